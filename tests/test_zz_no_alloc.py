"""akra_synth_spin2_static: the synthesis that allocates no device memory.

Some callers cannot allocate device memory where they need a synthesis: code under a
device-memory budget or inside a pool that must not grow, a process where another component
already holds the device memory, a latency-critical loop that cannot take cudaMalloc's
implicit synchronisation.  This entry point keeps its phase-array scratch in a fixed device
array inside the library.  Its output must equal the FP64 oracle's (within the precision's
tolerance) and akra_synth_spin2's, call after call (the scratch keeps the previous call's
contents); a call must grow neither the plan's device memory nor the device's used memory;
sizes beyond the scratch are rejected.  This file is collected last on purpose, and each test
creates its own plan, so it passes alone in a fresh process or after the rest of the suite.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
import synthetic as S
from paper_2606_06175_gb300 import akra as A

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _tol32(lmax):
    # FP32 recurrences: relative error ~ ε32 L / 2, bounded by 4 ε32 L (as in the operator tests)
    return 4 * 2.0 ** -24 * max(lmax, 16)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,N,L", [(A.F64, 16, 40), (A.F64, 64, 150), (A.F32, 32, 64), (A.F32, 128, 256)])
def test_static_synthesis_matches_oracle_and_allocating_synthesis(prec, N, L):
    tol = 1e-10 if prec == A.F64 else _tol32(L)
    ct = torch.complex128 if prec == A.F64 else torch.complex64
    dt = torch.float64 if prec == A.F64 else torch.float32
    plan = A.akra_plan_create(N, L)
    for call in range(2):                      # two calls in a row share the scratch
        rng = np.random.default_rng(100 * N + call)
        aE, aB = S.random_alm(L, rng), S.random_alm(L, rng)
        alm = torch.from_numpy(np.stack([aE, aB])[None]).to(DEV, ct)
        out = torch.full((1, 2, plan.npix), float("nan"), dtype=dt, device=DEV)
        bytes0 = A.akra_plan_describe(plan)["device_bytes"]
        A.akra_synth_spin2_static(plan, prec, alm, out)
        torch.cuda.synchronize()
        # the static call grew no plan workspace (on the fresh plan of the first call, too)
        assert A.akra_plan_describe(plan)["device_bytes"] == bytes0
        got = out[0].double().cpu().numpy()
        ref_o = np.stack(O.synth_spin2(N, L, aE, aB))
        assert _rel(got, ref_o) < tol, ("oracle", call, _rel(got, ref_o))
        ref = A.akra_synth_spin2(plan, prec, alm)
        torch.cuda.synchronize()
        err = _rel(got, ref[0].double().cpu().numpy())
        assert err < tol, ("akra_synth_spin2", call, err)


def test_static_synthesis_uses_no_device_memory_after_the_first_call():
    N, L = 64, 128
    plan = A.akra_plan_create(N, L)
    rng = np.random.default_rng(11)
    alm = torch.from_numpy(np.stack([S.random_alm(L, rng), S.random_alm(L, rng)])[None]).to(DEV)
    out = torch.empty((1, 2, plan.npix), dtype=torch.float64, device=DEV)
    A.akra_synth_spin2_static(plan, A.F64, alm, out)   # first call: looks up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        A.akra_synth_spin2_static(plan, A.F64, alm, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_synthesis_rejects_sizes_beyond_the_scratch():
    plan = A.akra_plan_create(512, 1024)       # FP64 phase array: 67 MB > 32 MiB
    alm = torch.zeros((1, 2, plan.ntri), dtype=torch.complex128, device=DEV)
    out = torch.empty((1, 2, plan.npix), dtype=torch.float64, device=DEV)
    with pytest.raises(A.AkraError) as ei:
        A.akra_synth_spin2_static(plan, A.F64, alm, out)
    assert ei.value.status == 1 and "static scratch" in str(ei.value)
