"""FP32 spin-2 Legendre synthesis with the l-contraction on the tcgen05 tensor core.

The recurrences run on the CUDA cores, their values split into a TF32 head and an FP32
remainder, and the contraction is three TF32 products accumulated in FP32.  Checked against
the FP64 oracle within the FP32 operator tolerance (4 ε32 lmax) for every RHS group size, with
RHS counts that leave the last group partly filled, on the synthesis alone (all rings, the
pure spin-2 transform), inside H on a masked sky, at a size with several tiles, chunks and a
ragged l-range, and inside mixed-precision solves (which must still converge to the FP64
solution)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
import synthetic as S
from paper_2606_06175_gb300 import akra as A

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def tol32(lmax):
    return 4 * 2.0 ** -24 * max(lmax, 16)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _alm(pairs):
    return torch.from_numpy(np.stack([np.stack(p) for p in pairs])).to(DEV, torch.complex64)


@pytest.mark.parametrize("group,R", [(4, 1), (4, 6), (8, 5), (16, 9), (32, 17)])
def test_tensor_synthesis_matches_oracle(group, R):
    N, L = 16, 45                      # several 16-step tiles, a ragged last one
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_tc_synthesis(p, R, group)
    assert A.akra_plan_get_tc_synthesis(p, R) == group
    rng = np.random.default_rng(group * 100 + R)
    pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
    g = A.akra_synth_spin2(p, A.F32, _alm(pairs)).double().cpu().numpy()
    for r in range(R):
        ref = np.stack(O.synth_spin2(N, L, *pairs[r]))
        assert rel(g[r], ref) < tol32(L), (group, R, r, rel(g[r], ref))


@pytest.mark.parametrize("group", [4, 8])
def test_tensor_synthesis_inside_H(group):
    N, L, R = 32, 64, 3
    p = A.akra_plan_create(N, L)
    rng = np.random.default_rng(5 + group)
    th, _ = O.pixel_angles(N)
    ninv = np.where(np.cos(th) < 0.3, 1.0 + rng.random(12 * N * N), 0.0)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    A.akra_plan_set_tc_synthesis(p, R, group)
    pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
    y = A.akra_apply_H(p, A.F32, _alm(pairs)).to(torch.complex128).cpu().numpy()
    w = O.Weights(N, ninv, 1e-3)
    for r in range(R):
        ref = np.stack(O.apply_H(N, L, w, *pairs[r]))
        assert rel(y[r], ref) < tol32(L), (group, r, rel(y[r], ref))


def test_tensor_synthesis_at_a_size_with_many_chunks_and_tiles():
    """Nside 128 / lmax 300: 256 ring pairs (2 chunks of 128 rows), 19 tiles, start points beyond
    the first tile for the polar pairs; sampled rings against the oracle's ring sums."""
    N, L = 128, 300
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_tc_synthesis(p, 1, 4)
    rng = np.random.default_rng(17)
    aE, aB = S.random_alm(L, rng), S.random_alm(L, rng)
    g = A.akra_synth_spin2(p, A.F32, _alm([(aE, aB)]))[0].double().cpu().numpy()
    ref = np.stack(O.synth_spin2(N, L, aE, aB))
    assert rel(g, ref) < tol32(L), rel(g, ref)


@pytest.mark.parametrize("R,group", [(1, 4), (4, 4)])
def test_mixed_solves_with_tensor_synthesis_reach_the_fp64_solution(R, group):
    wl = S.workload("cap32")
    N, L = wl["nside"], wl["lmax"]
    p = A.akra_plan_create(N, L)
    ninv = torch.from_numpy(wl["ninv"]).to(DEV)
    A.akra_plan_set_weights(p, ninv, 1e-3)
    A.akra_plan_set_tc_synthesis(p, R, group)
    xt = torch.from_numpy(np.stack(wl["x_true"])[None]).to(DEV).repeat(R, 1, 1)
    y = A.akra_apply_A(p, A.F64, xt)
    y += torch.from_numpy(wl["noise"][None]).to(DEV)
    y *= (ninv > 0).to(y.dtype)
    x64, i64 = A.akra_cg_solve(p, A.F64, y, tol=1e-11, maxiter=3000)
    xm, im = A.akra_cg_solve(p, A.MIXED, y, tol=1e-9, maxiter=3000)
    assert i64["status"] == 0 and im["status"] == 0, (i64, im)
    err = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
    assert err < 1e-6, err
