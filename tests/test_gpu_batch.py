"""The batched form (rbd_batch_* through the C ABI): many matrices of different sizes, tolerances
and modes in one persistent launch, each against the FP64 oracle on the same stored values.

Bar per matrix (float-float dot products, as the plain form): identical d and pivots; Y, T, err
and nu within 1e-10 (normwise), in cases whose steps keep nu / ||x_i|| above ~1e-3 (the two
sides' rounding is amplified by ||x_i|| / nu at each step and compounds over the steps; see
test_gpu_precision.py).  Also: the autotuned launch shape matches the default one to the bar,
a tuned run captured in a CUDA graph and replayed gives the same bits, tile rows and ring depth
leave every bit unchanged, a non-finite matrix fails alone, and the full 2048-matrix workload on
sampled matrices.
"""
import numpy as np
import pytest
import torch

import gen
from gpu_util import to_device, to_numpy

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def rbd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as pkg
    pkg.load()
    return pkg


def _parity(Xs, ref, c, what):
    scale = np.linalg.norm(Xs, axis=0)
    assert c.d == ref["d"], f"{what}: d {c.d} != {ref['d']}"
    assert np.array_equal(c.pivots.cpu().numpy(), ref["pivots"]), f"{what}: pivots"
    if c.d == 0:
        return
    assert np.linalg.norm(to_numpy(c.Y) - ref["Y"], axis=0).max() <= TOL, what
    assert (np.abs(to_numpy(c.T) - ref["T"]) / np.maximum(scale, 1e-300)[None, :]).max() <= TOL, what
    assert np.abs(c.err.cpu().numpy() - ref["err"]).max() <= TOL * scale.max(), what
    assert np.abs(c.nu.cpu().numpy() - ref["nu"]).max() <= TOL * scale.max(), what


def mixed_batch(dtype, seed):
    """Ragged shapes (rows not multiples of 4 or 128, single columns, d_max = min(m, n)), all three
    tolerance modes, nonzero start columns."""
    rng = np.random.default_rng(seed)
    shapes = [(100, 37), (256, 64), (777, 333), (1500, 20), (4000, 90), (129, 1), (1000, 700), (3001, 257),
              (64, 64), (2048, 150), (513, 513), (333, 1200)]
    items, host = [], []
    for i, (m, n) in enumerate(shapes):
        r = min(m, n)
        s = 2.0 ** (-np.arange(r) / (3 + i % 4)) * (1 + 0.5 * rng.random(r))
        X = gen.lowrank_haar(m, n, np.sort(s)[::-1], seed=seed * 100 + i, noise_sigma=1e-7)
        Xd = to_device(np.asfortranarray(X), dtype)
        mode = ("maxcol_rel", "fro_rel", "maxcol_abs")[i % 3]
        tol = {"maxcol_rel": 1e-3, "fro_rel": 1e-3, "maxcol_abs": 1e-3 * np.linalg.norm(X, axis=0).max()}[mode]
        d_max = min(m, n, 40 + 7 * i)
        items.append({"X": Xd, "tol": tol, "tol_mode": mode, "d_max": d_max, "start": (7 * i) % n})
        host.append(to_numpy(Xd))
    return items, host


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["fp32", "fp64"])
def test_batch_matches_oracle(rbd, oracle_mod, dtype):
    items, host = mixed_batch(dtype, 11 if dtype == torch.float32 else 12)
    plan = rbd.BatchPlan(items)
    plan.run()
    res = plan.results()
    for i, it in enumerate(items):
        assert res[i]["status"] == 0, i
        ref = oracle_mod.compress(host[i], it["tol"], it["d_max"], it["start"], it["tol_mode"])
        _parity(host[i], ref, plan.compressed(i, res[i]), f"matrix {i} {host[i].shape}")


def test_batch_equals_single_matrix_path(rbd):
    items, host = mixed_batch(torch.float32, 13)
    plan = rbd.BatchPlan(items)
    plan.run()
    res = plan.results()
    for i, it in enumerate(items):
        c = plan.compressed(i, res[i])
        s = rbd.compress(it["X"], it["tol"], it["d_max"], start=it["start"], tol_mode=it["tol_mode"])
        assert c.d == s.d and torch.equal(c.pivots, s.pivots), i
        if c.d:
            assert (c.Y - s.Y).abs().max().item() <= TOL
            scale = torch.linalg.vector_norm(it["X"].double(), dim=0).max().item()
            assert (c.T - s.T).abs().max().item() <= TOL * scale


def _snapshot(plan):
    torch.cuda.synchronize()
    return plan.res.clone(), [(o["T"].clone(), o["Y"].clone(), o["pivots"].clone()) for o in plan.out], plan.results()


def _same_bits(plan, snap):
    res, outs, _ = snap
    assert torch.equal(plan.res, res)
    for i, (o, (T, Y, piv)) in enumerate(zip(plan.out, outs)):
        d = plan.results()[i]["d"]
        assert torch.equal(o["T"][:d], T[:d]) and torch.equal(o["Y"][:, :d], Y[:, :d]), i
        assert torch.equal(o["pivots"][:d], piv[:d]), i


def _close(plan, snap, items):
    """The same d and pivots, Y and T within the parity bar (a launch shape regroups sums)."""
    _, outs, ref = snap
    got = plan.results()
    for i, (o, (T, Y, piv)) in enumerate(zip(plan.out, outs)):
        d = got[i]["d"]
        assert d == ref[i]["d"] and got[i]["status"] == 0, i
        assert torch.equal(o["pivots"][:d], piv[:d]), i
        scale = torch.linalg.vector_norm(items[i]["X"].double(), dim=0).max().item()
        assert (o["Y"][:, :d] - Y[:, :d]).abs().max().item() <= TOL, i
        assert (o["T"][:d] - T[:d]).abs().max().item() <= TOL * scale, i


def test_tuned_plan_and_graph_replay(rbd, tmp_path):
    """The autotuner's choice (group width, tile rows, team size, ring depth) is kept in the plan
    and in the JSON cache under the batch's bucket; the tuned plan matches the default one to the
    parity bar, and a run of it captured in a CUDA graph and replayed gives its exact bits."""
    items, _ = mixed_batch(torch.float32, 14)
    plan = rbd.BatchPlan(items)
    assert plan.config() == {"cols": 16, "tile_rows": 256, "team_pct": 150, "stages": plan.config()["stages"]}
    plan.run()
    default = _snapshot(plan)
    cache = str(tmp_path / "tune.json")
    cfg = plan.tune(cache=cache)
    assert not cfg["cached"]
    assert cfg["cols"] in (16, 32) and cfg["tile_rows"] in (128, 256) and cfg["team_pct"] in (75, 150, 300)
    assert cfg["stages"] >= 2
    assert plan.config() == {k: cfg[k] for k in ("cols", "tile_rows", "team_pct", "stages")}
    plan.run()
    tuned = _snapshot(plan)
    _close(plan, default, items)
    for o in plan.out:
        o["T"].zero_()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.run()  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        plan.run()
    for o in plan.out:
        o["T"].zero_()
    g.replay()
    _same_bits(plan, tuned)
    # a second plan over the same batch takes the cached shape without timing
    plan2 = rbd.BatchPlan(items)
    cfg2 = plan2.tune(cache=cache)
    assert cfg2["cached"] and {k: cfg2[k] for k in plan2.config()} == plan2.config()
    plan2.run()
    _same_bits(plan2, tuned)


def test_every_launch_shape_matches(rbd):
    """Every launch shape gives the default plan's d and pivots and its Y and T to the parity bar;
    the tile rows and ring depth alone leave every bit unchanged."""
    items, _ = mixed_batch(torch.float64, 16)
    plan = rbd.BatchPlan(items)
    plan.run()
    default = _snapshot(plan)
    for cols in (16, 32):
        for team in (75, 150, 300):
            base = None
            for rows in (256, 128):
                for stages in (0, 2):
                    plan.set_config({"cols": cols, "tile_rows": rows, "team_pct": team, "stages": stages})
                    plan.run()
                    _close(plan, default, items)
                    if base is None:
                        base = _snapshot(plan)
                    else:
                        _same_bits(plan, base)
    with pytest.raises(rbd.RbdError):
        plan.set_config({"cols": 24, "tile_rows": 256, "team_pct": 150})


def test_nonfinite_matrix_fails_alone(rbd, oracle_mod):
    items, host = mixed_batch(torch.float64, 15)
    bad = items[3]["X"].clone()
    bad[5, 2] = float("nan")
    items[3] = dict(items[3], X=bad)
    plan = rbd.BatchPlan(items)
    plan.run()
    res = plan.results()
    assert res[3]["status"] == 4 and res[3]["d"] == 0
    for i in (0, 1, 2, 4, 5):
        assert res[i]["status"] == 0
        ref = oracle_mod.compress(host[i], items[i]["tol"], items[i]["d_max"], items[i]["start"],
                                  items[i]["tol_mode"])
        _parity(host[i], ref, plan.compressed(i, res[i]), f"matrix {i}")


def test_batch_limits_rejected(rbd):
    X = torch.zeros((10, 5000), dtype=torch.float32, device="cuda").t()
    with pytest.raises(rbd.RbdError) as ei:
        rbd.BatchPlan([{"X": X, "tol": 0.0, "d_max": 4}])
    assert ei.value.status == 6  # RBD_EUNSUPPORTED: more than 4096 rows


def test_batched_workload_2048_sampled(rbd, oracle_mod):
    """The batched workload: 2048 FP32 matrices, m log-uniform in [256, 4096], n in [64, 2048],
    s_i = exp(-r i) (r ~ U[0.05, 0.5], truncated at 1e-9), tol log-uniform in [1e-6, 1e-2]
    (relative max-column), d_max = min(m, n, 512).  Eight sampled matrices against the oracle;
    every matrix: status, stop rule, and the certified indicator under its tolerance."""
    specs = gen.batch_specs(2048, seed=3)
    items = []
    for sp in specs:
        s = gen.decay_spectrum(sp["rate"], min(sp["m"], sp["n"]))
        X = gen.lowrank_torch(sp["m"], sp["n"], s, sp["seed"], device="cuda", dtype=torch.float32)
        items.append({"X": X, "tol": sp["tol"], "tol_mode": "maxcol_rel", "d_max": sp["d_max"],
                          "d_hint": sp["d_hint"]})
    plan = rbd.BatchPlan(items)
    plan.run()
    res = plan.results()
    for i, r in enumerate(res):
        assert r["status"] == 0, i
        assert r["stop_reason"] in (1, 2, 3), i
        if r["stop_reason"] == 1:
            assert r["err_last"] <= items[i]["tol"] * r["x_maxcol"], i
    rng = np.random.default_rng(0)
    for i in rng.choice(len(items), 8, replace=False):
        Xs = to_numpy(items[i]["X"])
        ref = oracle_mod.compress(Xs, items[i]["tol"], items[i]["d_max"], 0, "maxcol_rel")
        c = plan.compressed(int(i), res[int(i)])
        # the well-conditioned prefix (nu / ||x_i|| >= 1e-3): identical pivots, values within the
        # bar; deeper steps approach the FP32 data's rounding noise, where the two sides' rounding,
        # amplified by ||x_i|| / nu and compounded over the steps, reaches the bar and pivot
        # choices between near-equal residuals are decided by rounding
        xn = np.linalg.norm(Xs, axis=0)
        ok = ref["nu"] / xn[ref["pivots"]] >= 1e-3
        kk = int(np.argmin(ok)) if not ok.all() else ref["d"]
        kk = min(kk, c.d)
        assert np.array_equal(c.pivots.cpu().numpy()[:kk], ref["pivots"][:kk]), int(i)
        if kk:
            assert np.linalg.norm(to_numpy(c.Y)[:, :kk] - ref["Y"][:, :kk], axis=0).max() <= TOL, int(i)
            assert (np.abs(to_numpy(c.T)[:kk] - ref["T"][:kk]) / xn[None, :]).max() <= TOL, int(i)
