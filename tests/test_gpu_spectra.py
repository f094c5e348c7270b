"""Noise-realisation pipeline (Sec. IV, "Power spectrum results"): the shuffling gather and the
E/B spectra against the oracle, and the whole pipeline (shuffle -> batched mixed solve ->
band powers) against the oracle's pipeline on the cap workload."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
import synthetic as S
from paper_2606_06175_gb300 import akra as A
from paper_2606_06175_gb300 import spectra as SP

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_shuffle_matches_oracle_bitwise():
    N = 16
    p = A.akra_plan_create(N, 32)
    rng = np.random.default_rng(3)
    mask = rng.random(12 * N * N) < 0.3
    y = np.where(mask, rng.normal(size=(2, 12 * N * N)), 0.0)
    perms = SP.shuffle_permutations(mask, 3, seed=1)
    for prec, dt in [(A.F64, torch.float64), (A.F32, torch.float32)]:
        out = A.akra_shuffle_shear(p, prec, torch.from_numpy(y).to(DEV, dt),
                                   torch.from_numpy(perms).to(DEV)).cpu().numpy()
        for r in range(3):
            ref = O.shuffle_shear(y.astype(np.float32) if prec == A.F32 else y, perms[r])
            assert np.array_equal(out[r], ref)
    bad = torch.from_numpy(perms[:1]).to(DEV)
    bad[0, 5] = 12 * N * N
    with pytest.raises(A.AkraError):
        A.akra_shuffle_shear(p, A.F64, torch.from_numpy(y).to(DEV), bad)


@pytest.mark.parametrize("L", [40, 301])
def test_cl_spectra_match_oracle(L):
    p = A.akra_plan_create(128, L)
    rng = np.random.default_rng(L)
    a = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(2)]
    b = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(2)]
    ta = torch.from_numpy(np.stack([np.stack(x) for x in a])).to(DEV)
    tb = torch.from_numpy(np.stack([np.stack(x) for x in b])).to(DEV)
    edges = np.geomspace(3, L, 6)
    for prec, tol in [(A.F64, 1e-12), (A.F32, 2e-6)]:
        xa = ta if prec == A.F64 else ta.to(torch.complex64)
        xb = tb if prec == A.F64 else tb.to(torch.complex64)
        cl = A.akra_cl_spectra(p, prec, xa, xb).cpu().numpy()
        bp = A.akra_cl_spectra(p, prec, xa, xb, edges=edges).cpu().numpy()
        auto = A.akra_cl_spectra(p, prec, xa).cpu().numpy()
        for r in range(2):
            ref = O.cl_spectra(L, a[r], b[r])
            assert np.max(np.abs(cl[r] - ref)) < tol * np.max(np.abs(ref))
            assert np.max(np.abs(bp[r] - O.band_powers(ref, edges))) < tol * np.max(np.abs(ref))
            ra = O.cl_spectra(L, a[r], a[r])
            assert np.max(np.abs(auto[r] - ra)) < tol * np.max(np.abs(ra))


def test_noise_realisation_pipeline_matches_oracle():
    wl = S.workload("cap32")
    N, L = wl["nside"], wl["lmax"]
    y = np.stack(O.forward_A(N, L, *wl["x_true"])) + wl["noise"]
    mask = wl["ninv"] > 0
    y = np.where(mask, y, 0.0)
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    perms = SP.shuffle_permutations(mask, 3, seed=77)
    edges = np.geomspace(2, L, 5)
    bp, xs, info = SP.noise_realisations(p, A.MIXED, torch.from_numpy(y).to(DEV), perms, edges=edges,
                                         tol=1e-9, maxiter=3000)
    assert info["status"] == 0 and info["relres"] < 1e-9
    bp = bp.cpu().numpy()
    w = O.Weights(N, wl["ninv"], 1e-3)
    for r in range(3):
        ys = O.shuffle_shear(y, perms[r])
        (xE, xB), _, _, _ = O.cg_solve(N, L, w, ys[0], ys[1], tol=1e-12, maxiter=3000)
        ref = O.band_powers(O.cl_spectra(L, (xE, xB), (xE, xB)), edges)
        # solutions agree to ~1e-6 (mixed at 1e-9), band powers are quadratic in them
        assert np.max(np.abs(bp[r] - ref)) < 1e-5 * np.max(np.abs(ref)), r
    mean, std = SP.noise_bias(torch.from_numpy(bp))
    assert mean.shape == (4, len(edges) - 1) and torch.all(std >= 0)
