"""Noise-realisation pipeline and power spectra (Sec. IV, "Power spectrum results").

The shape-noise bias N_l of an auto spectrum is estimated from reconstructions of shuffled
catalogues: the observed shear values are permuted among the unmasked pixels (survey geometry
and noise level kept, signal correlations destroyed), every shuffled map goes through the full
reconstruction, and the mean auto spectrum of those maps is N_l.  Here the shuffled maps are the
RHS of one batched solve; shuffling, solving and spectra run in the library's kernels.  The
permutations are drawn on the host from a seeded generator and passed in (the library draws no
random numbers).
"""
from __future__ import annotations

import numpy as np
import torch

from . import akra as A

# 8 logarithmic bins over 10 < l <= 1024 (the band-power binning of the differentiation workload)
DEFAULT_EDGES = tuple(np.geomspace(10, 1024, 9))


def shuffle_permutations(mask: np.ndarray, nreal: int, seed: int) -> np.ndarray:
    """[nreal, npix] int32 source pixels: a uniform random permutation of the unmasked pixels
    onto themselves, masked pixels mapped to themselves."""
    mask = np.asarray(mask, bool)
    rng = np.random.default_rng(seed)
    idx = np.nonzero(mask)[0]
    out = np.tile(np.arange(mask.size, dtype=np.int32), (nreal, 1))
    for r in range(nreal):
        out[r, idx] = idx[rng.permutation(idx.size)]
    return out


def noise_realisations(plan: A.Plan, prec: int, shear: torch.Tensor, perms: np.ndarray, edges=DEFAULT_EDGES,
                       tol: float = 1e-6, maxiter: int = 2000):
    """Shuffle `shear` [2, npix] with each permutation, reconstruct all of them in one batched
    solve and return (band powers [nreal, 4, nbins] (EE, EB, BE, BB auto), solved alm, solve info)."""
    mprec = A.F32 if prec == A.F32 else A.F64
    p = torch.from_numpy(np.ascontiguousarray(perms, np.int32)).to(shear.device)
    ys = A.akra_shuffle_shear(plan, mprec, shear.contiguous(), p)
    xs, info = A.akra_cg_solve(plan, prec, ys, tol=tol, maxiter=maxiter)
    bp = A.akra_cl_spectra(plan, mprec, xs, edges=edges)
    return bp, xs, info


def noise_bias(bp: torch.Tensor):
    """Mean and standard deviation over realisations of the shuffled maps' band powers."""
    bp = bp.double()
    return bp.mean(dim=0), (bp.std(dim=0) if bp.shape[0] > 1 else torch.zeros_like(bp[0]))
