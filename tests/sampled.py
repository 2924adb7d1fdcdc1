"""Checks of large GPU runs on outputs the oracle can compute one by one."""
import numpy as np

import oracle


def _keys(R):
    """Rows (tx, rx, n, types..., labels...) with entries past n set to a sentinel."""
    n = R["n"].astype(np.int64)
    q = np.arange(R["type"].shape[1])[None, :]
    live = q < n[:, None]
    t = np.where(live, R["type"], -1).astype(np.int64)
    lab = np.where(live, R["label"].astype(np.int64), -1)
    return np.column_stack([R["tx"], R["rx"], n, t, lab]), t


def _limits(t, p):
    assert ((t == 0).sum(axis=1) <= p.max_refl).all()
    assert ((t == 1).sum(axis=1) <= p.max_diff).all()


def coarse_invariants(C, p):
    """kappa per (TX, RX, types, labels) and the interaction limits of every coarse path."""
    assert C["counts"]["overflow"] == 0
    rows, t = _keys(C)
    _limits(t, p)
    if len(rows):
        _, cnt = np.unique(rows, axis=0, return_counts=True)
        assert cnt.max() <= p.kappa


def exact_invariants(F, p):
    """One exact path per (TX, RX, types, labels), within the interaction limits."""
    rows, t = _keys(F)
    _limits(t, p)
    if len(rows):
        _, cnt = np.unique(rows, axis=0, return_counts=True)
        assert cnt.max() == 1
    assert (F["status"] == 0).all() and (F["length"] > 0).all()


def sampled_refinement(sc, C, A, osc, n, seed, min_agree=0.95, min_both=20):
    """n sampled coarse paths refined by the oracle one by one: status agreement,
    interaction points within 1e-3 m and lengths within 1e-6 relative."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(C["n"]), size=min(n, len(C["n"])), replace=False))
    sub = {k: C[k][idx] for k in ("tx", "rx", "n", "ie", "type", "label")}
    R = osc.refine_given(sc.tx, sc.rx, sub)
    g_status = A["status"][idx]
    agree = g_status == R["status"]
    assert agree.mean() >= min_agree, (g_status, R["status"])
    both = np.where((g_status == 0) & (R["status"] == 0))[0]
    assert len(both) >= min_both
    for j in both:
        m = int(sub["n"][j])
        np.testing.assert_allclose(A["pts"][idx[j]][:m], R["pts"][j][:m], atol=1e-3)
        assert abs(A["length"][idx[j]] - R["length"][j]) <= 1e-6 * R["length"][j]
    return agree.mean(), len(both)


def sampled_visibility(sc, C, osc, n, seed, min_frac=0.97):
    """Each segment of n sampled coarse paths passes the oracle's visibility test."""
    ies = osc.ies()
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(C["n"]), size=min(n, len(C["n"])), replace=False)
    ok = total = 0
    for i in idx:
        m = int(C["n"][i])
        nodes = [(sc.tx[C["tx"][i]], 0, oracle.NONE_LABEL)]
        for q in range(m):
            ie = int(C["ie"][i][q])
            nodes.append((ies["rp"][ie], 2 if ies["kind"][ie] == 1 else 1, int(ies["label"][ie])))
        nodes.append((sc.rx[C["rx"][i]], 0, oracle.NONE_LABEL))
        for (a, ma, la), (b, mb, lb) in zip(nodes[:-1], nodes[1:]):
            total += 1
            ok += osc.visible(a, b, ma, la, mb, lb)
    assert ok >= min_frac * total
    return ok / max(total, 1)
