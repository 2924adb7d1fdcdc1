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


def oracle_confirms(osc, sc, P, i, p, IGN_LABEL=1, IGN_ANY=2):
    """Path i of P checked against the definition of an exact path on the oracle's
    scene osc (Section 2.3): every reflection point on its label's Eq. 1 surface,
    every diffraction point on its edge, the length stationary (the norm over all
    interactions of e_in + e_out projected on the tangent plane of Eq. 1's normal, or
    on the edge direction), and every segment visible under the endpoint rules.
    Returns (largest |f| or distance off the edge, gradient norm, all visible)."""
    from oracle import NONE_LABEL
    n = int(P["n"][i])
    nodes = [np.asarray(sc.tx[P["tx"][i]], float)] + [np.asarray(x, float) for x in P["pts"][i][:n]] + \
        [np.asarray(sc.rx[P["rx"][i]], float)]
    ies = osc.ies() if n and (np.asarray(P["type"][i][:n]) == 1).any() else None
    f_max = 0.0
    g2 = 0.0
    for k in range(n):
        x = nodes[k + 1]
        e = (x - nodes[k]) / np.linalg.norm(x - nodes[k]) + (x - nodes[k + 2]) / np.linalg.norm(x - nodes[k + 2])
        if int(P["type"][i][k]) == 0:
            f, nn = osc.sdf_label(int(P["label"][i][k]), x)
            if f is None:
                return np.inf, np.inf, False
            f_max = max(f_max, abs(f))
            g2 += float(e @ e - (e @ nn) ** 2)
        else:
            ed = sc.edges[ies["edge"][int(P["ie"][i][k])]]
            p0, p1 = ed[:3], ed[3:6]
            w = (p1 - p0) / np.linalg.norm(p1 - p0)
            off = (x - p0) - ((x - p0) @ w) * w
            f_max = max(f_max, float(np.linalg.norm(off)))
            g2 += float(e @ w) ** 2
    vis = True
    for k in range(n + 1):
        ma, la = (0, NONE_LABEL) if k == 0 else (
            IGN_ANY if int(P["type"][i][k - 1]) == 1 else IGN_LABEL, int(P["label"][i][k - 1]))
        mb, lb = (0, NONE_LABEL) if k == n else (
            IGN_ANY if int(P["type"][i][k]) == 1 else IGN_LABEL, int(P["label"][i][k]))
        vis = vis and osc.visible(nodes[k], nodes[k + 1], ma, la, mb, lb)
    return f_max, float(np.sqrt(max(g2, 0.0))), vis


def confirm_alternates(G, bad, sc, p, max_bad):
    """The paths of G that differ from the oracle's winner of their label sequence
    (compare's `bad`) are alternate stationary points: at most max_bad of them, each
    confirmed by the oracle as an exact path (oracle_confirms) and within 1e-4
    relative length of the oracle's winner.  On the noisy cloud one coarse path's
    gradient descent can settle on one of several stationary points, or cycle around
    one until rho, and which candidate wins the shortest-path dedup can depend on
    rounding."""
    assert len(bad) <= max_bad, bad[:5]
    if not bad:
        return
    import oracle
    osc = oracle.Scene.from_scene(sc, p)
    where = {}
    for i in range(len(G["n"])):
        n = int(G["n"][i])
        where[(int(G["tx"][i]), int(G["rx"][i]), tuple(int(t) for t in G["type"][i][:n]),
               tuple(int(l) for l in G["label"][i][:n]))] = i
    for key, dp, dl in bad:
        f_max, grad, vis = oracle_confirms(osc, sc, G, where[key], p)
        assert f_max < 1e-4 and grad < p.delta and vis, (key, dp, dl, f_max, grad, vis)
        assert dl < 1e-4, (key, dp, dl)
