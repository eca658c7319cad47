"""Batched form: heterogeneous completions advanced by one graph per iteration.

Every instance must end exactly where the same context run alone ends (the
kernels, their data and their reduction orders are the same; only the
concurrency differs), across the tuning trials and after the choice, and one
instance is checked against the oracle.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import method as O

pytestmark = pytest.mark.gpu

SETTING = (1e-3, 1e-3, 1e-1)
CASES = [  # precision, shape, r, observed
    ("fp64", (16, 48, 7), 2, 0.5),
    ("fp32", (20, 40, 112), 4, 0.3),
    ("fp32", (24, 36, 168), 8, 0.2),
    ("fp64", (9, 30, 12), 3, 0.4),
    ("fp32", (30, 50, 28), 5, 0.3),
    ("fp32", (12, 24, 8), 3, 0.6),
    ("tf32", (200, 96, 12), 32, 0.3),   # tensor cores, the X-step's graph branch
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09838_gb300 import build
    build.build()


def _ctx(precision, shape, r, obs, seed):
    from paper_2005_09838_gb300 import tc
    w = wl.custom(*shape, r, obs, seed=seed)
    inst = wl.generate(w)
    dt = np.float64 if precision == "fp64" else np.float32
    if precision != "fp64":
        inst = wl.as_precision(inst, np.float32)
    prec = {"fp64": tc.TC_FP64, "fp32": tc.TC_FP32, "tf32": tc.TC_TF32}[precision]
    p = tc.make_params(*shape, r, *SETTING, precision=prec)
    c = tc.Completion(p, wl.to_colmajor(inst["G"], dt), wl.to_colmajor(inst["mask"], np.uint8),
                      wl.to_colmajor(inst["Y0"], dt))
    return c, inst


def test_batched_instances_match_their_solo_runs():
    from paper_2005_09838_gb300 import tc
    batched, solo, insts = [], [], []
    for q, (prec, shape, r, obs) in enumerate(CASES):
        a, inst = _ctx(prec, shape, r, obs, 6000 + q)
        b, _ = _ctx(prec, shape, r, obs, 6000 + q)
        batched.append(a)
        solo.append(b)
        insts.append(inst)
    with tc.Batch(batched) as B:
        B.iterate(3)          # tuning trials: every one is a real iteration of all instances
        assert B.branches() == 0
        B.iterate(5)
        assert B.branches() in (1, 4, len(CASES))
        n0, loop = B.launches()
        assert loop == 1      # after the trials, the device-side loop
        B.iterate(2)          # the chosen graph: two iterations in one launch
        B.iterate(7)
        n1, _ = B.launches()
        assert n1 - n0 == 2
    for c in solo:
        c.iterate(17)
    for (prec, shape, r, obs), a, b in zip(CASES, batched, solo):
        Wa, _, _ = a.result_numpy()
        Wb, _, _ = b.result_numpy()
        assert np.array_equal(Wa, Wb), (prec, shape)
        assert a.objective()[0] == b.objective()[0]
    # the transform tile chosen at init: 2, 4 or 8 for generic lengths, 0 where a
    # dedicated kernel exists (7, 112, 168 in FP32; 7 in FP64)
    for (prec, shape, r, obs), a in zip(CASES, batched):
        dedicated = shape[2] == 7 or (prec != "fp64" and shape[2] in (112, 168))
        assert (a.tile() == 0) if dedicated else (a.tile() in (2, 4, 8)), (prec, shape, a.tile())
    # and the oracle agrees with one of them
    prec, shape, r, _ = CASES[0]
    ref = O.tctf2r(insts[0]["G"], insts[0]["mask"], r, *SETTING, insts[0]["Y0"], iters=17)
    W0, _, _ = batched[0].result_numpy()
    W0 = wl.from_colmajor(W0, shape)
    assert np.linalg.norm(W0 - ref["W"]) <= 1e-10 * np.linalg.norm(ref["W"])
    for c in batched + solo:
        c.close()


def test_batch_rejects_bad_arguments():
    from paper_2005_09838_gb300 import tc
    a, _ = _ctx("fp32", (12, 24, 8), 3, 0.5, 6100)
    with pytest.raises(tc.TCError) as ei:
        tc.Batch([a, a])
    assert "TC_ERR_ARG" in str(ei.value)
    a.close()
