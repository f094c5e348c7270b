"""Several instances (uneven Nside / lmax, several RHS each) in one batched solve.

Checks: the batched FP32 H of every instance against the FP64 oracle's H (tol32); batched
mixed-precision and FP32 solves against the oracle's FP64 solutions; the autotuner; and the
uneven-instance workload at its own sizes (32 noise realisations at Nside 1024 / lmax 2048,
16 at 512 / 1024, 16 at 256 / 512, DES-like footprint): every RHS converges to 1e-6 and
agrees with the single-plan solve of the same RHS.
"""
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


SMALL = [(8, 16, 3), (16, 40, 2), (32, 64, 1)]


def _small_instances(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for N, L, R in SMALL:
        th, ph = O.pixel_angles(N)
        ninv = np.where((th > 0.8) & (np.cos(2 * ph) > -0.8), rng.poisson(25, 12 * N * N) / 0.26 ** 2, 0.0)
        p = A.akra_plan_create(N, L)
        A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
        out.append((N, L, R, ninv, p))
    return out, rng


def test_batched_H_matches_oracle():
    inst, rng = _small_instances(1)
    plans = [p for *_, p in inst]
    b = A.akra_batch_create(plans, [R for _, _, R, _, _ in inst])
    xs, refs = [], []
    for N, L, R, ninv, p in inst:
        pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
        xs.append(torch.from_numpy(np.stack([np.stack(q) for q in pairs])).to(DEV, torch.complex64))
        w = O.Weights(N, ninv, 1e-3)
        refs.append([np.stack(O.apply_H(N, L, w, *q)) for q in pairs])
    ys = A.akra_batch_apply_H(b, xs)
    for (N, L, R, _, _), y, ref in zip(inst, ys, refs):
        yn = y.to(torch.complex128).cpu().numpy()
        for r in range(R):
            assert rel(yn[r], ref[r]) < tol32(L), (N, L, r)
    # the autotuner keeps a compiled shape and the batched H still agrees
    A.akra_batch_autotune(b)
    d = A.akra_batch_describe(b)
    assert (d["P"], d["RG"]) in {(1, 4), (2, 2), (1, 2), (4, 1), (5, 1), (6, 1), (2, 1)}
    ys2 = A.akra_batch_apply_H(b, xs)
    for (N, L, R, _, _), y, ref in zip(inst, ys2, refs):
        yn = y.to(torch.complex128).cpu().numpy()
        for r in range(R):
            assert rel(yn[r], ref[r]) < tol32(L)


@pytest.mark.parametrize("group", [4, 8, 16, 32])
def test_batched_H_with_tensor_synthesis_matches_oracle(group):
    """The batch's synthesis on the tensor cores (persistent queue over 128-pair chunks and RHS
    groups of every size; R = 5, 9, 3 leave the last group of each instance partly filled)."""
    rng = np.random.default_rng(40 + group)
    spec = [(8, 16, 5), (32, 70, 9), (16, 40, 3)]
    plans, xs, refs = [], [], []
    for N, L, R in spec:
        th, ph = O.pixel_angles(N)
        ninv = np.where((th > 0.5) & (np.cos(2 * ph) > -0.8), 1.0 + rng.random(12 * N * N), 0.0)
        p = A.akra_plan_create(N, L)
        A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
        pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
        xs.append(torch.from_numpy(np.stack([np.stack(q) for q in pairs])).to(DEV, torch.complex64))
        w = O.Weights(N, ninv, 1e-3)
        refs.append([np.stack(O.apply_H(N, L, w, *q)) for q in pairs])
        plans.append(p)
    b = A.akra_batch_create(plans, [R for *_, R in spec])
    A.akra_batch_set_tc_synthesis(b, group)
    assert A.akra_batch_get_tc_synthesis(b) == group
    for _ in range(2):   # the second pass reuses the blocks' TMEM and barriers across items
        ys = A.akra_batch_apply_H(b, xs)
        for (N, L, R), y, ref in zip(spec, ys, refs):
            yn = y.to(torch.complex128).cpu().numpy()
            for r in range(R):
                assert rel(yn[r], ref[r]) < tol32(L), (group, N, L, r, rel(yn[r], ref[r]))
    A.akra_batch_set_tc_synthesis(b, 0)
    ys = A.akra_batch_apply_H(b, xs)
    for (N, L, R), y, ref in zip(spec, ys, refs):
        yn = y.to(torch.complex128).cpu().numpy()
        assert max(rel(yn[r], ref[r]) for r in range(R)) < tol32(L)
    with pytest.raises(A.AkraError):
        A.akra_batch_set_tc_synthesis(b, 12)


def test_batched_mixed_solve_with_tensor_synthesis():
    inst, rng = _small_instances(3)
    b = A.akra_batch_create([p for *_, p in inst], [R for _, _, R, _, _ in inst])
    A.akra_batch_set_tc_synthesis(b, 4)
    shears, refs = [], []
    for N, L, R, ninv, p in inst:
        ys = []
        for _ in range(R):
            kE = S.random_alm(L, rng, lmin=2) * 0.05
            y = np.stack(O.forward_A(N, L, kE, np.zeros_like(kE))) + 0.01 * rng.normal(size=(2, 12 * N * N))
            ys.append(np.where(ninv > 0, y, 0.0))
        w = O.Weights(N, ninv, 1e-3)
        refs.append([np.stack(O.cg_solve(N, L, w, y[0], y[1], tol=1e-12, maxiter=5000)[0]) for y in ys])
        shears.append(torch.from_numpy(np.stack(ys)).to(DEV, torch.float64))
    xs, infos = A.akra_batch_cg_solve(b, A.MIXED, shears, tol=1e-9, maxiter=5000)
    for (N, L, R, _, _), x, ref, info in zip(inst, xs, refs, infos):
        assert info["status"] == 0 and info["relres"] < 1e-9, info
        xn = x.to(torch.complex128).cpu().numpy()
        for r in range(R):
            assert rel(xn[r], ref[r]) < 1e-6, (N, L, r)


@pytest.mark.parametrize("prec", [A.MIXED, A.F32])
def test_batched_solve_matches_oracle(prec):
    inst, rng = _small_instances(2)
    b = A.akra_batch_create([p for *_, p in inst], [R for _, _, R, _, _ in inst])
    shears, refs = [], []
    for N, L, R, ninv, p in inst:
        ys = []
        for _ in range(R):
            kE = S.random_alm(L, rng, lmin=2) * 0.05
            y = np.stack(O.forward_A(N, L, kE, np.zeros_like(kE))) + 0.01 * rng.normal(size=(2, 12 * N * N))
            ys.append(np.where(ninv > 0, y, 0.0))
        w = O.Weights(N, ninv, 1e-3)
        refs.append([np.stack(O.cg_solve(N, L, w, y[0], y[1], tol=1e-12, maxiter=5000)[0]) for y in ys])
        shears.append(torch.from_numpy(np.stack(ys)).to(DEV, torch.float64 if prec == A.MIXED else torch.float32))
    tol = 1e-9 if prec == A.MIXED else 1e-5
    xs, infos = A.akra_batch_cg_solve(b, prec, shears, tol=tol, maxiter=5000)
    for (N, L, R, _, _), x, ref, info in zip(inst, xs, refs, infos):
        assert info["status"] == 0, info
        xn = x.to(torch.complex128).cpu().numpy()
        # FP32 end to end: solution error up to ~κ ε32 sqrt(L) (κ ~ 1e3 on these small masks)
        for r in range(R):
            e = rel(xn[r], ref[r])
            assert e < (1e-6 if prec == A.MIXED else 2e-2), (N, L, r, e)
        if prec == A.MIXED:
            assert info["outer"] >= 1 and info["relres"] < tol


def test_uneven_instances_workload():
    """32 noise realisations at (1024, 2048), 16 at (512, 1024), 16 at (256, 512)."""
    spec = [(1024, 2048, 32), (512, 1024, 16), (256, 512, 16)]
    plans, shears, ninvs = [], [], []
    for k, (N, L, R) in enumerate(spec):
        sv = S.survey(N, "des", S.SEEDS["batch"] + k)
        p = A.akra_plan_create(N, L)
        A.akra_plan_set_weights(p, torch.from_numpy(sv["ninv"]).to(DEV), 1e-3)
        noise = S.shape_noise(sv["ninv"], sv["rng_noise"], nreal=R)
        plans.append(p)
        ninvs.append(sv["ninv"])
        shears.append(torch.from_numpy(noise).to(DEV))
    b = A.akra_batch_create(plans, [R for *_, R in spec])
    A.akra_batch_autotune(b)
    xs, infos = A.akra_batch_cg_solve(b, A.MIXED, shears, tol=1e-6, maxiter=3000)
    for info in infos:
        assert info["status"] == 0 and max(info["relres_rhs"]) < 1e-6, info
    # every RHS's FP64 residual recomputed with the single-plan operators (not the batch kernels)
    for (N, L, R), p, y, x in zip(spec, plans, shears, xs):
        _, ms = O.lm_arrays(L)
        w = torch.from_numpy(np.where(ms == 0, 1.0, 2.0)).to(DEV)
        m0 = torch.from_numpy(ms == 0).to(DEV)
        bvec = A.akra_apply_At(p, A.F64, y, weighted=True)
        r = bvec - A.akra_apply_H(p, A.F64, x)

        def n2(v):
            vi = torch.where(m0, 0.0, v.imag)
            return (w * (v.real ** 2 + vi ** 2)).sum(dim=(-1, -2))

        relres = torch.sqrt(n2(r) / n2(bvec))
        assert float(relres.max()) < 1.05e-6, (N, L, relres.max())
