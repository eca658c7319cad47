"""Step 5 of the TCTF2R Algorithm (rank vector) on the GPU against the oracle.

The data are t-products whose factor A has one column constant along mode 3,
so the DC slice has rank 3 and every other slice rank 2 (plus 1% noise).
With the rank rule on (tc_rank_rule: drop the directions whose Y-step Gram
eigenvalue stays at or below tol * lambda_max for `patience` iterations), the
GPU must reach the oracle's rank vector (oracle.tctf2r_rank) and match its W
and f0 within the FP64 / FP32 bars.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import method as O

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09838_gb300 import build
    build.build()


def _data(m1, m2, m3, obs, seed, precision):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m1, 3, m3))
    B = rng.standard_normal((3, m2, m3))
    A[:, 2, :] = A[:, 2, :1]
    T = O.tprod_definition(A, B)
    M = T + 0.01 * math.sqrt(float(np.mean(T * T))) * rng.standard_normal(T.shape)
    mask = rng.random(T.shape) < obs
    Y0 = rng.standard_normal((3, m2, m3))
    if precision == "fp32":
        M, Y0 = (a.astype(np.float32).astype(np.float64) for a in (M, Y0))
    return M, np.where(mask, M, 0.0), mask, Y0


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fully_observed_slices_drop_to_their_data_rank(precision):
    # fully observed: W = G, so the fit itself is compared, through f0 and the
    # observed residual ||Z - G||
    from paper_2005_09838_gb300 import api
    M, G, mask, Y0 = _data(40, 60, 8, 1.0, 7, precision)
    setting = (0.0, 1e-3, 0.0)
    ref = O.tctf2r_rank(G, mask, 3, *setting, Y0, iters=15, rank_tol=1e-2, patience=2)
    got = api.complete(G, mask, Y0, 3, 15, *setting, precision=precision, rank_tol=1e-2, rank_patience=2)
    assert got["ranks"] == ref["ranks"] == [3, 2, 2, 2, 2, 2, 2, 2]
    assert abs(got["f0"] - ref["f0"]) <= TOL[precision] * abs(ref["f0"])
    resid_ref = float(np.linalg.norm(ref["Z"] - G))
    assert abs(got["resid_obs"] - resid_ref) <= TOL[precision] * resid_ref


@pytest.mark.parametrize("precision,m3", [("fp64", 8), ("fp32", 8), ("fp32", 112)])
def test_partially_observed_rank_rule_matches_oracle(precision, m3):
    # 60% observed, setting R: the slices settle at rank 2 (the DC slice at 3);
    # n3 = 112 runs the shared-memory transform of the slab kernel
    from paper_2005_09838_gb300 import api
    M, G, mask, Y0 = _data(40, 60, m3, 0.6, 7, precision)
    setting = (1e-3, 1e-3, 1e-1)
    ref = O.tctf2r_rank(G, mask, 3, *setting, Y0, iters=20, rank_tol=0.08, patience=2)
    got = api.complete(G, mask, Y0, 3, 20, *setting, precision=precision, rank_tol=0.08, rank_patience=2)
    print(f"{precision} n3={m3}: ranks {got['ranks'][:6]}..., W {_rel(got['W'], ref['W']):.2e}")
    assert got["ranks"] == ref["ranks"]
    assert _rel(got["W"], ref["W"]) <= TOL[precision]
    assert abs(got["f0"] - ref["f0"]) <= TOL[precision] * abs(ref["f0"])
    assert abs(wl.nmse(M, got["W"], mask) - wl.nmse(M, ref["W"], mask)) <= 1e-4


def test_rule_off_keeps_the_ranks_reached():
    # tc_rank_rule(0) after some adjustments: the ranks stay, the iteration
    # continues at those ranks (the oracle: the same run with the rule, whose
    # ranks have settled, then more iterations)
    from paper_2005_09838_gb300 import tc
    M, G, mask, Y0 = _data(40, 60, 8, 1.0, 7, "fp64")
    p = tc.make_params(40, 60, 8, 3, 0.0, 1e-3, 0.0, precision=tc.TC_FP64)
    with tc.Completion(p, wl.to_colmajor(G), wl.to_colmajor(mask, np.uint8), wl.to_colmajor(Y0)) as c:
        assert c.ranks() == [3] * 8
        c.rank_rule(1e-2, 2)
        c.iterate(10)
        before = c.ranks()
        c.rank_rule(0.0)
        c.iterate(5)
        assert c.ranks() == before == [3, 2, 2, 2, 2, 2, 2, 2]
        f_gpu, _ = c.objective()
    ref = O.tctf2r_rank(G, mask, 3, 0.0, 1e-3, 0.0, Y0, iters=15, rank_tol=1e-2, patience=2)
    assert ref["ranks"] == before
    assert abs(f_gpu - ref["f0"]) <= TOL["fp64"] * abs(ref["f0"])
