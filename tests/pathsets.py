"""Helpers that compare path sets from the CUDA library and the oracle."""
import numpy as np


def keyed(P):
    """{(tx, rx, types, labels): (points (n,3), length)} of a path dict."""
    out = {}
    for i in range(len(P["n"])):
        n = int(P["n"][i])
        key = (int(P["tx"][i]), int(P["rx"][i]), tuple(int(t) for t in P["type"][i][:n]),
               tuple(int(l) for l in P["label"][i][:n]))
        assert key not in out, f"duplicate path {key}"
        out[key] = (np.array(P["pts"][i][:n], dtype=np.float64), float(P["length"][i]))
    return out


def compare(gpu, ref, atol_pts=1e-3, rtol_len=1e-6):
    """Counts of matched paths and the worst point / length errors over them."""
    g, r = keyed(gpu), keyed(ref)
    common = g.keys() & r.keys()
    worst_pt = 0.0
    worst_len = 0.0
    bad = []
    for k in common:
        dp = float(np.abs(g[k][0] - r[k][0]).max()) if len(k[2]) else 0.0
        dl = abs(g[k][1] - r[k][1]) / max(r[k][1], 1e-12)
        worst_pt = max(worst_pt, dp)
        worst_len = max(worst_len, dl)
        if dp > atol_pts or dl > rtol_len:
            bad.append((k, dp, dl))
    union = g.keys() | r.keys()
    return dict(n_gpu=len(g), n_ref=len(r), n_common=len(common), only_gpu=sorted(g.keys() - r.keys()),
                only_ref=sorted(r.keys() - g.keys()), worst_pt=worst_pt, worst_len=worst_len, bad=bad,
                jaccard=len(common) / max(1, len(union)))
