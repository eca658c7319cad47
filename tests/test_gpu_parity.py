"""GPU parity of the TCTF2R path against the FP64 oracle (same seeded inputs).

Tolerances (relative Frobenius error on W, and relative error on f0):
FP64 path 1e-10, FP32 path 1e-5; recovery NMSE within 1e-4 of the oracle's.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import method as O

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}
SETTINGS = {"R": (1e-3, 1e-3, 1e-1), "B": (0.0, 0.0, 0.0)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09838_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _run_pair(w, setting, precision, iters, inst=None, want_factors=False):
    from paper_2005_09838_gb300 import api
    inst = inst or wl.generate(w)
    if precision == "fp32":
        inst = wl.as_precision(inst, np.float32)
    mu, rho1, rho2 = SETTINGS[setting] if isinstance(setting, str) else setting
    ref = O.tctf2r(inst["G"], inst["mask"], w.r, mu, rho1, rho2, inst["Y0"], iters=iters)
    got = api.complete(inst["G"], inst["mask"], inst["Y0"], w.r, iters, mu, rho1, rho2, precision,
                       want_factors=want_factors)
    return inst, ref, got


@pytest.mark.parametrize("setting", ["R", "B"])
def test_c1_fp64_full_trajectory(setting):
    w = wl.c1()
    inst, ref, got = _run_pair(w, setting, "fp64", w.iters, want_factors=True)
    assert _rel(got["W"], ref["W"]) <= TOL["fp64"]
    assert abs(got["f0"] - ref["f0"]) <= TOL["fp64"] * abs(ref["f0"])
    assert abs(got["resid_obs"] - ref["resid_obs"]) <= 1e-8 * max(ref["resid_obs"], 1.0)
    # same trajectory: the spatial factors agree too
    assert _rel(got["X"], ref["X"]) <= 1e-8
    assert _rel(got["Y"], ref["Y"]) <= 1e-8
    assert abs(wl.nmse(inst["M"], got["W"], inst["mask"]) - wl.nmse(inst["M"], ref["W"], inst["mask"])) <= 1e-4


@pytest.mark.parametrize("shape,r,obs", [
    ((20, 40, 112), 4, 0.3),    # register FFT n3 = 112, several warps, ragged n2
    ((37, 100, 168), 8, 0.2),   # register FFT n3 = 168, ragged n1 and n2
])
@pytest.mark.parametrize("setting", ["R", "B"])
def test_fp32_specialised_lengths(shape, r, obs, setting):
    w = wl.custom(*shape, r, obs, seed=1000 + shape[2] + r, iters=25)
    inst, ref, got = _run_pair(w, setting, "fp32", w.iters)
    assert _rel(got["W"], ref["W"]) <= TOL["fp32"]
    assert abs(got["f0"] - ref["f0"]) <= TOL["fp32"] * abs(ref["f0"])
    assert abs(wl.nmse(inst["M"], got["W"], inst["mask"]) - wl.nmse(inst["M"], ref["W"], inst["mask"])) <= 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("n3", [1, 2, 9, 12])
def test_generic_lengths(precision, n3):
    w = wl.custom(11, 35, n3, 3, 0.4, seed=2000 + n3, iters=12)
    inst, ref, got = _run_pair(w, "R", precision, w.iters)
    assert _rel(got["W"], ref["W"]) <= TOL[precision]
    assert abs(got["f0"] - ref["f0"]) <= TOL[precision] * abs(ref["f0"])


@pytest.mark.parametrize("setting", [(0.2, 0.5, 3.0), (0.0, 0.0, 0.7)])
def test_strong_regularisation_fp64(setting):
    w = wl.custom(9, 30, 7, 2, 0.3, seed=77, iters=20)
    inst, ref, got = _run_pair(w, setting, "fp64", w.iters)
    assert _rel(got["W"], ref["W"]) <= TOL["fp64"]
    assert abs(got["f0"] - ref["f0"]) <= TOL["fp64"] * abs(ref["f0"])


def test_degenerate_masks_fp64():
    # fully observed rows, fully missing rows, a fully missing frontal slice,
    # and r = 1
    w = wl.custom(8, 33, 7, 1, 0.5, seed=5, iters=10)
    inst = wl.generate(w)
    mask = inst["mask"].copy()
    mask[0, :, :] = True
    mask[1, :, :] = False
    mask[:, :, 3] = False
    mask[:, 0, :] = False
    mask[:, -1, :] = True
    inst["mask"] = mask
    inst["G"] = np.where(mask, inst["M"], 0.0)
    _, ref, got = _run_pair(w, "R", "fp64", w.iters, inst=inst)
    assert _rel(got["W"], ref["W"]) <= TOL["fp64"]


@pytest.mark.parametrize("n3", [112, 168])
def test_degenerate_masks_fp32_shared_memory_transform(n3):
    # the same run boundaries through the FP32 slab kernel with the
    # shared-memory transform and the table-driven W-step: fully observed and
    # fully missing OD rows, a missing frontal slice, j = 0 always missing and
    # j = n2 - 1 always observed, ragged n2 (two mask words), r = 1
    w = wl.custom(8, 37, n3, 1, 0.5, seed=5 + n3, iters=10)
    inst = wl.as_precision(wl.generate(w), np.float32)
    mask = inst["mask"].copy()
    mask[0, :, :] = True
    mask[1, :, :] = False
    mask[:, :, 3] = False
    mask[:, 0, :] = False
    mask[:, -1, :] = True
    inst["mask"] = mask
    inst["G"] = np.where(mask, inst["M"], 0.0)
    _, ref, got = _run_pair(w, "R", "fp32", w.iters, inst=inst)
    assert _rel(got["W"], ref["W"]) <= TOL["fp32"]
    assert abs(got["f0"] - ref["f0"]) <= TOL["fp32"] * abs(ref["f0"])


def test_fully_observed_exact_rank_recovery_fp64():
    # Proposition "tubrank": exact low-tubal-rank data, fully observed
    rng = np.random.default_rng(3)
    A = rng.standard_normal((10, 2, 7))
    B = rng.standard_normal((2, 16, 7))
    T = O.tprod_definition(A, B)
    from paper_2005_09838_gb300 import api
    got = api.complete(T, np.ones(T.shape, bool), rng.standard_normal((2, 16, 7)), 2, 30, precision="fp64")
    # W = G on the mask; the model X*Y reproduces T: ||P_Omega(Z - G)|| ~ 0
    assert got["resid_obs"] <= 1e-10 * np.linalg.norm(T)


def test_objective_is_monotone_fp32():
    # Theorem "GlobConvergM": f0 non-increasing along the iteration
    from paper_2005_09838_gb300 import tc
    w = wl.custom(24, 48, 112, 4, 0.3, seed=9, iters=1)
    inst = wl.as_precision(wl.generate(w), np.float32)
    p = tc.make_params(w.n1, w.n2, w.n3, w.r, 1e-3, 1e-3, 1e-1, precision=tc.TC_FP32)
    g = wl.to_colmajor(inst["G"], np.float32)
    m = wl.to_colmajor(inst["mask"], np.uint8)
    y = wl.to_colmajor(inst["Y0"], np.float32)
    with tc.Completion(p, g, m, y) as c:
        prev = np.inf
        for _ in range(30):
            c.iterate(1)
            f, _ = c.objective()
            assert f <= prev * (1 + 1e-5)
            prev = f


def test_iterate_zero_and_repeat_calls_fp64():
    # tc_iterate(a) then tc_iterate(b) equals tc_iterate(a + b)
    from paper_2005_09838_gb300 import tc
    w = wl.custom(6, 20, 7, 2, 0.5, seed=11)
    inst = wl.generate(w)
    p = tc.make_params(w.n1, w.n2, w.n3, w.r, 1e-3, 1e-3, 1e-1, precision=tc.TC_FP64)
    args = (wl.to_colmajor(inst["G"]), wl.to_colmajor(inst["mask"], np.uint8), wl.to_colmajor(inst["Y0"]))
    with tc.Completion(p, *args) as a, tc.Completion(p, *args) as b:
        a.iterate(0)
        a.iterate(3)
        a.iterate(4)
        b.iterate(7)
        wa, _, _ = a.result_numpy()
        wb, _, _ = b.result_numpy()
        np.testing.assert_array_equal(wa, wb)


def test_device_inputs_match_host_inputs_fp32():
    import torch
    from paper_2005_09838_gb300 import tc
    w = wl.custom(16, 64, 112, 4, 0.3, seed=12)
    inst = wl.as_precision(wl.generate(w), np.float32)
    p = tc.make_params(w.n1, w.n2, w.n3, w.r, 1e-3, 1e-3, 1e-1, precision=tc.TC_FP32)
    g = wl.to_colmajor(inst["G"], np.float32)
    m = wl.to_colmajor(inst["mask"], np.uint8)
    y = wl.to_colmajor(inst["Y0"], np.float32)
    dg, dm, dy = (torch.from_numpy(a).cuda() for a in (g, m, y))
    stream = torch.cuda.current_stream().cuda_stream
    with tc.Completion(p, g, m, y) as a, tc.Completion(p, dg, dm, dy, on_device=True, stream=stream) as b:
        a.iterate(5)
        b.iterate(5)
        wa, _, _ = a.result_numpy()
        Wd = torch.empty(w.N, dtype=torch.float32, device="cuda")
        b.result(Wd, on_device=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(wa, Wd.cpu().numpy())


def test_c2_full_size_three_iterations_fp32():
    # the bench workload (144 x 288 x 168, r = 8, 20% observed), first three
    # iterations of the trajectory against the oracle
    w = wl.c2(0.2)
    inst, ref, got = _run_pair(w, "R", "fp32", 3)
    assert _rel(got["W"], ref["W"]) <= TOL["fp32"]
    assert abs(got["f0"] - ref["f0"]) <= TOL["fp32"] * abs(ref["f0"])


@pytest.mark.parametrize("precision,n1", [("fp32", 1000), ("fp64", 700)])
def test_rank32_longest_slices(precision, n1):
    # r = 32 with long slices (n1 = 1000 / 700): B = QA^+ over eight 128-row
    # chunks per slice, the column update and Gram partials over many chunks
    w = wl.custom(n1, 40, 8, 32, 0.3, seed=3200 + n1, iters=6)
    inst, ref, got = _run_pair(w, "R", precision, w.iters)
    assert _rel(got["W"], ref["W"]) <= TOL[precision]
    assert abs(got["f0"] - ref["f0"]) <= TOL[precision] * abs(ref["f0"])


@pytest.mark.parametrize("r", [12, 16])
def test_fp32_middle_ranks(r):
    # 8 < r <= 16 in an FP32 engine: the X-step spread over the GPU with the
    # r <= 16 layout of the B = QA^+ tiles (four column groups per warp) and the
    # r x r solves in FP32 storage; n1 = 150 (two ragged 128-row chunks)
    w = wl.custom(150, 48, 12, r, 0.4, seed=4100 + r, iters=8)
    inst, ref, got = _run_pair(w, "R", "fp32", w.iters)
    assert _rel(got["W"], ref["W"]) <= TOL["fp32"]
    assert abs(got["f0"] - ref["f0"]) <= TOL["fp32"] * abs(ref["f0"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_rank32_long_slices(precision):
    # r = 32 (block Gauss-Jordan pseudo-inverse) with n1 = 529: the FP32 Y-step
    # cannot stage the 32 x 529 slice of X~ and reads it from global memory
    w = wl.custom(529, 40, 12, 32, 0.3, seed=3100, iters=8)
    inst, ref, got = _run_pair(w, "R", precision, w.iters)
    assert _rel(got["W"], ref["W"]) <= TOL[precision]
    assert abs(got["f0"] - ref["f0"]) <= TOL[precision] * abs(ref["f0"])


def test_c3_full_size_three_iterations_fp32():
    # the precision-form workload (529 x 96 x 112, r = 32, 30% observed) in
    # plain FP32, first three iterations against the oracle.  The Gram
    # X~'^H H_rho1 X~' of the DC slice has condition number 1.5e4 - 3.6e4 over
    # these iterations: its FP64 pseudo-inverse is applied in FP64 (real-slice
    # path of the FP32 engine)
    w = wl.c3(0.3)
    inst, ref, got = _run_pair(w, "R", "fp32", 3)
    print(f"C3 FP32: W {_rel(got['W'], ref['W']):.2e}, f0 {abs(got['f0'] - ref['f0']) / abs(ref['f0']):.2e}")
    assert _rel(got["W"], ref["W"]) <= TOL["fp32"]
    assert abs(got["f0"] - ref["f0"]) <= TOL["fp32"] * abs(ref["f0"])
