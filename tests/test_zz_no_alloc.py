"""akra_synth_spin2_static: the synthesis that allocates no device memory.

For callers that cannot allocate at the point of the call (inside a stream capture, under
an allocation budget, in latency-critical loops): the phase-array scratch is a fixed device
array inside the library.  Its output must equal akra_synth_spin2's, call after call (the
scratch keeps the previous call's contents), and sizes beyond the scratch are rejected.
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from paper_2606_06175_gb300 import akra as A

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _alm(L, seed, prec):
    rng = np.random.default_rng(seed)
    arr = np.stack([S.random_alm(L, rng), S.random_alm(L, rng)])[None]
    return torch.from_numpy(arr).to(DEV, torch.complex128 if prec == A.F64 else torch.complex64)


@pytest.mark.parametrize("prec,N,L,tol", [(A.F64, 16, 40, 1e-10), (A.F64, 64, 150, 1e-10),
                                          (A.F32, 32, 64, 1e-5), (A.F32, 128, 256, 1e-5)])
def test_static_synthesis_equals_allocating_synthesis(prec, N, L, tol):
    plan = A.akra_plan_create(N, L)
    dt = torch.float64 if prec == A.F64 else torch.float32
    for call in range(2):                      # two calls in a row share the scratch
        alm = _alm(L, 100 * N + call, prec)
        ref = A.akra_synth_spin2(plan, prec, alm)
        out = torch.full((1, 2, plan.npix), float("nan"), dtype=dt, device=DEV)
        A.akra_synth_spin2_static(plan, prec, alm, out)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
        assert err < tol, (call, err)


def test_static_synthesis_rejects_sizes_beyond_the_scratch():
    plan = A.akra_plan_create(512, 1024)       # FP64 phase array: 67 MB > 32 MiB
    alm = torch.zeros((1, 2, plan.ntri), dtype=torch.complex128, device=DEV)
    out = torch.empty((1, 2, plan.npix), dtype=torch.float64, device=DEV)
    with pytest.raises(A.AkraError) as ei:
        A.akra_synth_spin2_static(plan, A.F64, alm, out)
    assert ei.value.status == 1 and "static scratch" in str(ei.value)
