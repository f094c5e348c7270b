"""Run by tests/test_gpu_debug_build.py in a child process whose AKRA_LIBRARY names the
bounds-checked build (libakra_debug.so): every operator family and solver at small sizes,
checked against the FP64 oracle, then the library's out-of-bounds record.  Prints one JSON line."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import oracle as O  # noqa: E402
import synthetic as S  # noqa: E402
from paper_2606_06175_gb300 import akra as A  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def main():
    dev = torch.device("cuda:0")
    out = {"library": os.path.basename(A.library_path()), "errors": {}}
    A.akra_debug_violations()   # start from a clear record
    for N, L, R in ((8, 20, 1), (16, 40, 2)):
        rng = np.random.default_rng(N)
        th, ph = O.pixel_angles(N)
        ninv = np.where((th > 1.0) & (ph < 5.0), rng.uniform(100, 300, 12 * N * N), 0.0)
        kE, kB = S.random_alm(L, rng, lmin=2), S.random_alm(L, rng, lmin=2)
        p = A.akra_plan_create(N, L)
        A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(dev), 1e-3)
        x = torch.from_numpy(np.repeat(np.stack([kE, kB])[None], R, 0)).to(dev)
        w = O.Weights(N, ninv, 1e-3)
        g = np.stack(O.synth_spin2(N, L, kE, kB))
        h = np.stack(O.apply_H(N, L, w, kE, kB))
        for prec, tol in ((A.F64, 1e-10), (A.F32, 4 * 2.0 ** -24 * 64)):
            xx = x if prec == A.F64 else x.to(torch.complex64)
            s = A.akra_synth_spin2(p, prec, xx)[R - 1].double().cpu().numpy()
            hh = A.akra_apply_H(p, prec, xx)[R - 1].to(torch.complex128).cpu().numpy()
            out["errors"]["synth_%d_%d" % (N, prec)] = rel(s, g)
            out["errors"]["H_%d_%d" % (N, prec)] = rel(hh, h)
            assert rel(s, g) < tol and rel(hh, h) < tol, (N, prec, rel(s, g), rel(hh, h))
        y = torch.from_numpy(np.repeat(np.where(ninv > 0, g, 0.0)[None], R, 0)).to(dev)
        for prec in (A.F64, A.MIXED):
            xs, info = A.akra_cg_solve(p, prec, y, tol=1e-8, maxiter=3000)
            assert info["status"] == 0, info
        xs32, info = A.akra_cg_solve(p, A.F32, y.float(), tol=1e-4, maxiter=3000)
        assert info["status"] == 0, info
        # the persistent work-queue kernels and the batched FFT, with the CUDA-core and the
        # tensor-core synthesis (its operand staging kernel and prefetch ring included)
        bt = A.akra_batch_create([p], [R])
        xb = x.to(torch.complex64)
        for group in (0, 4):
            A.akra_batch_set_tc_synthesis(bt, group)
            yb = A.akra_batch_apply_H(bt, [xb])[0]
            e = rel(yb[R - 1].to(torch.complex128).cpu().numpy(), h)
            out["errors"]["batch_H_%d_tc%d" % (N, group)] = e
            assert e < 4 * 2.0 ** -24 * 64, (N, group, e)
        del bt
        # the single-plan tensor-core synthesis, RHS groups partly filled
        for group in (4, 8):
            A.akra_plan_set_tc_synthesis(p, R, group)
            s = A.akra_synth_spin2(p, A.F32, x.to(torch.complex64))[R - 1].double().cpu().numpy()
            out["errors"]["synth_tc%d_%d" % (group, N)] = rel(s, g)
            assert rel(s, g) < 4 * 2.0 ** -24 * 64, (N, group, rel(s, g))
    torch.cuda.synchronize()
    out["violations"] = A.akra_debug_violations()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
