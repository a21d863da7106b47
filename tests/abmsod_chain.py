"""Per-iteration comparison of an ABMSOD implementation with the plain
binary64 oracle (Alg. 2, Eq. 6 and 7).

The oracle's own search is replayed one iteration at a time: from each
state (x_t, H_t) it visits, one oracle iteration gives (x_{t+1}, H_{t+1},
rho_{t+1}), and the implementation under test runs one iteration from the
same state.  Inputs flow only from the oracle to the implementation, so a
difference in one iteration cannot carry into the next.

Bounds for one iteration (the implementation sums binary32 terms on
fixed-point grids; the oracle evaluates the definition in binary64):
  - every iteration: |dx'| <= 2.5e-4 voxel (x' comes from the window at
    the given state, whose membership both sides decide exactly);
  - iterations whose window at x' has no counted voxel within 2^-18 of the
    boundary, relative to |o|^T |H^-1| |o| (far beyond what a centre that
    differs by the x' bound can move): the same window voxels,
    |dH| <= 5e-4 max(1, max_a H_aa), |drho| <= 5e-6, and the same stopping
    decision wherever |rho' - best| > 5e-6;
  - other iterations (a voxel of the window at x' on its boundary up to the
    x' difference, where either side may count it): window voxels within
    1% + 4, |dH| <= 0.05 max(1, max_a H_aa), |drho| <= 5e-3.
"""
import numpy as np

EDGE = 2.0 ** -18
TOL_X, TOL_H, TOL_RHO = 2.5e-4, 5e-4, 5e-6
NEAR_H, NEAR_RHO = 0.05, 5e-3


def seed_items(seeds, r_min, r_max):
    """(x, H) of every (seed, r) item, seed-major, H = r^2 I."""
    seeds = np.asarray(seeds, np.float64).reshape(-1, 3)
    S = r_max - r_min + 1
    x = np.repeat(seeds, S, 0)
    r2 = np.tile(np.arange(r_min, r_max + 1, dtype=np.float64) ** 2, len(seeds))
    H = np.zeros((len(x), 6))
    H[:, 0] = H[:, 3] = H[:, 5] = r2
    return x, H


def oracle_states(ko, bins, B, x0, H0, max_iter):
    """Replay the oracle's searches from (x0, H0) one iteration at a time.
    Returns the states each iteration starts from and the oracle's one-
    iteration results there, plus the best rho before the iteration."""
    x = np.array(x0, np.float64)
    H = np.array(H0, np.float64)
    n = len(x)
    best = np.zeros(n)
    alive = np.ones(n, bool)
    parts = []
    for t in range(max_iter):
        idx = np.nonzero(alive)[0]
        if len(idx) == 0:
            break
        o = ko.abmsod(bins, B, 0, 0, None, 1, cand=(x[idx], H[idx]))
        done = o["iters"] == 1           # an empty window ends the search early
        parts.append({"x": x[idx][done], "H": H[idx][done], "xn": o["x"][done],
                      "Hn": o["H"][done], "rho": o["rho"][done], "edge": o["edge"][done],
                      "voxels": o["voxels"][done], "best": best[idx][done],
                      "item": idx[done], "t": np.full(int(done.sum()), t)})
        fell = o["rho"] < best[idx]
        go = done & ~fell
        x[idx[go]] = o["x"][go]
        H[idx[go]] = o["H"][go]
        best[idx] = np.maximum(best[idx], np.where(done, o["rho"], 0.0))
        alive[idx[~go]] = False
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def compare(states, got):
    """Check one-iteration results `got` (fields x (n, 3), H (n, 6), rho,
    voxels, iters) from the states' starts against the oracle's results at
    the bounds above.  Returns (iterations checked strictly, near-edge)."""
    assert np.all(got["iters"] == 1)
    far = states["edge"] > EDGE
    Hs = np.maximum(1.0, states["Hn"][:, [0, 3, 5]].max(1))
    dx = np.abs(got["x"] - states["xn"]).max(1)
    dH = np.abs(got["H"] - states["Hn"]).max(1) / Hs
    dr = np.abs(got["rho"] - states["rho"])
    dv = np.abs(got["voxels"].astype(np.int64) - states["voxels"])

    def report(mask, what):
        i = np.nonzero(mask)[0][:3]
        return f"{mask.sum()} iterations {what}; first items {states['item'][i]} t {states['t'][i]}"

    assert not (far & (dv != 0)).any(), report(far & (dv != 0), "count other window voxels")
    assert not (dx > TOL_X).any(), report(dx > TOL_X, f"|dx| > {TOL_X}")
    assert not (far & (dH > TOL_H)).any(), report(far & (dH > TOL_H), f"|dH| > {TOL_H}")
    assert not (far & (dr > TOL_RHO)).any(), report(far & (dr > TOL_RHO), f"|drho| > {TOL_RHO}")
    decided = far & (np.abs(states["rho"] - states["best"]) > TOL_RHO)
    fell_o = states["rho"] < states["best"]
    fell_g = got["rho"] < states["best"]
    assert not (decided & (fell_o != fell_g)).any(), report(decided & (fell_o != fell_g),
                                                            "take another stopping decision")
    near = ~far
    vb = 0.01 * states["voxels"] + 4
    assert not (near & (dv > vb)).any(), report(near & (dv > vb), "differ in many voxels")
    assert not (near & (dH > NEAR_H)).any(), report(near & (dH > NEAR_H), f"|dH| > {NEAR_H}")
    assert not (near & (dr > NEAR_RHO)).any(), report(near & (dr > NEAR_RHO),
                                                      f"|drho| > {NEAR_RHO}")
    return int(far.sum()), int(near.sum())
