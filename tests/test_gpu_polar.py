"""A footprint that reaches a pole: the 30-degree cap of the small workload moved to dec -85 deg,
at Nside 512 / lmax 1024 (the ring pairs within 0.1 rad of the pole run the FP32 recurrence in
difference form).  The mixed solve must converge with as few outer FP64 steps as on the DES-like
footprint, and run below the κ-scaled bound its solution must be within 1e-6 of the FP64 GPU
solution; the FP32 synthesis on the polar rings must meet the FP32 operator tolerance."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
import synthetic as S
from paper_2606_06175_gb300 import akra as A

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N, L = 512, 1024


def tol32(lmax):
    return 4 * 2.0 ** -24 * max(lmax, 16)


@pytest.fixture(scope="module")
def polar():
    z, phi = S.pixel_positions(N)
    fp = S.cap_footprint(z, phi, radius_deg=30.0, dec0_deg=-85.0, ra0_deg=30.0)
    rng = np.random.default_rng(85)
    counts = np.where(fp, rng.poisson(5.6 * S.pixel_area_arcmin2(N), size=fp.shape), 0)
    ninv = np.where(counts > 0, counts / S.SIGMA_E ** 2, 0.0)
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    kE = S.grf_alm(L, S.cl_kappa(L), rng)
    xt = torch.from_numpy(np.stack([kE, np.zeros_like(kE)])[None]).to(DEV)
    y = A.akra_apply_A(p, A.F64, xt)
    sd = np.where(ninv > 0, 1.0 / np.sqrt(np.where(ninv > 0, ninv, 1.0)), 0.0)
    y += torch.from_numpy((rng.standard_normal((2, ninv.size)) * sd)[None]).to(DEV)
    y *= torch.from_numpy(ninv > 0).to(DEV)
    return p, y, ninv


def test_polar_cap_mixed_solve_against_fp64(polar):
    p, y, ninv = polar
    assert float(np.min(S.pixel_positions(N)[0][ninv > 0])) < -0.9999   # the footprint reaches the pole
    x64, i64 = A.akra_cg_solve(p, A.F64, y, tol=1e-10, maxiter=5000)
    xm6, im6 = A.akra_cg_solve(p, A.MIXED, y, tol=1e-6, maxiter=5000)
    xm8, im8 = A.akra_cg_solve(p, A.MIXED, y, tol=1e-8, maxiter=5000)
    assert i64["status"] == 0 and im6["status"] == 0 and im8["status"] == 0
    # as on the DES-like footprint: two outer steps (three FP64 applications) reach 1e-6
    assert im6["outer"] <= 2 and im6["h_applies_f64"] <= 3, im6
    err = float(torch.linalg.vector_norm(xm8 - x64) / torch.linalg.vector_norm(x64))
    assert err < 1e-6, err


def test_polar_rings_fp32_synthesis(polar):
    p = polar[0]
    rng = np.random.default_rng(3)
    aE, aB = S.random_alm(L, rng), S.random_alm(L, rng)
    g = A.akra_synth_spin2(p, A.F32, torch.from_numpy(np.stack([aE, aB])[None]).to(DEV, torch.complex64))[0]
    rings = np.array([1, 2, 3, 5, 9, 17, 40, 2047, 2046, 2040], np.int32)
    F = O.legendre_synth(N, L, aE, aB, rings)
    for k, r in enumerate(rings):
        ct, st, n, sg, first = O.ring_info(N, int(r))
        ref = O.ring_phase_sum(F[k], L, n, sg)
        got = g[:, first:first + n].double().cpu().numpy()
        err = math.sqrt(float((np.abs(got[0] + 1j * got[1] - ref) ** 2).sum()) / float((np.abs(ref) ** 2).sum()))
        assert err < tol32(L), (int(r), err)
