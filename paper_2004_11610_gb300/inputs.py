"""Seeded synthetic inputs for the extra-component apply.

This module holds random-vector and workload recipes only; it contains none of
the method's arithmetic, so the CUDA path and the FP64 oracle can both be fed
from it.  The paper applies its matrices to random vectors (Section 5.1:
vectors of i.i.d. uniform numbers); the workloads below reproduce those shapes
with fixed seeds.

Seeds: base seed 2004, plus the workload index, plus a plan index.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 2004

# Family names shared by the binding, the tests and the oracle's callers.
FAMILIES = ("chebyshev", "legendre", "jacobi", "laguerre", "hermite")


def rng(*offsets: int) -> np.random.Generator:
    """A PCG64 generator seeded from the base seed plus the given offsets."""
    return np.random.default_rng([BASE_SEED, *[int(o) for o in offsets]])


def uniform_pm1(n: int, nrhs: int, *offsets: int) -> np.ndarray:
    """nrhs vectors of length n with i.i.d. uniform[-1, 1) entries, shape (nrhs, n)."""
    return rng(*offsets).uniform(-1.0, 1.0, size=(nrhs, n))


def uniform_01(n: int, nrhs: int, *offsets: int) -> np.ndarray:
    """nrhs vectors with i.i.d. uniform[0, 1) entries (the paper's Section 5.1 input)."""
    return rng(*offsets).uniform(0.0, 1.0, size=(nrhs, n))


def normal(n: int, nrhs: int, *offsets: int) -> np.ndarray:
    """nrhs vectors with i.i.d. standard-normal entries, shape (nrhs, n)."""
    return rng(*offsets).standard_normal(size=(nrhs, n))


def complex_normal(n: int, nrhs: int, *offsets: int) -> np.ndarray:
    """nrhs complex vectors whose real and imaginary parts are i.i.d. standard
    normal (the imaginary parts from the stream offset by 1000)."""
    return normal(n, nrhs, *offsets) + 1j * normal(n, nrhs, *(tuple(offsets) + (1000,)))


# Named workloads.  Each entry gives the plans (family, N, parameters), the
# tolerance threshold eps, the precision of the apply, the number of
# right-hand sides and the input distribution.
WORKLOADS = {
    # Legendre at N=512 Gauss-Legendre nodes, plain FP64, eps=1e-14, one RHS.
    "legendre512_fp64": dict(
        plans=[("legendre", 512, {})], eps=1e-14, precision="fp64", nrhs=1, dist="uniform_pm1"),
    # Chebyshev T at 4096 Chebyshev-Gauss points and Laguerre functions at 4096
    # Gauss-Laguerre nodes, FP64, eps=1e-12, 64 standard-normal RHS.
    "cheb_lag4096_fp64": dict(
        plans=[("chebyshev", 4096, {}), ("laguerre", 4096, {})], eps=1e-12, precision="fp64",
        nrhs=64, dist="normal"),
    # The same workload with FP64 vectors and FFTs but the band products in
    # FP32 pairs (XC_FP64_PAIR).
    "cheb_lag4096_fp64pair": dict(
        plans=[("chebyshev", 4096, {}), ("laguerre", 4096, {})], eps=1e-12, precision="fp64pair",
        nrhs=64, dist="normal"),
    # Legendre and Jacobi(1/2,-1/2) at N=16384, FP32 compensated apply,
    # eps=1e-7, 256 uniform[-1,1] RHS.
    "leg_jac16384_fp32c": dict(
        plans=[("legendre", 16384, {}), ("jacobi", 16384, {"alpha": 0.5, "beta": -0.5})],
        eps=1e-7, precision="fp32c", nrhs=256, dist="uniform_pm1"),
    # Legendre at N=32768, FP32 forward and adjoint, 128 standard-normal RHS.
    "legendre32768_fp32": dict(
        plans=[("legendre", 32768, {})], eps=1e-7, precision="fp32", nrhs=128, dist="normal"),
    # Complex families: exp(i m theta_n) at the 8192 arc-midpoint angles, and
    # the spectral Laguerre matrix with the shape parameters of the paper's
    # Section 4 figure (eta = 2500, T = 4 s) at N = 8192; FP64, eps=1e-12, 64
    # complex standard-normal RHS.
    "exp8192_fp64": dict(
        plans=[("exp", 8192, {})], eps=1e-12, precision="fp64", nrhs=64, dist="complex_normal"),
    "lagspec8192_fp64": dict(
        plans=[("lagspec", 8192, {"alpha": 2500.0, "beta": 4.0})], eps=1e-12, precision="fp64", nrhs=64,
        dist="complex_normal"),
    # The Laguerre transform matrix of Section 5.3 (Laguerre functions at the
    # equispaced points eta t_i, t_i = 12 (i+1)/(N-1), eta = 100) under the
    # 2-D block scheme, N = 4096, eps=1e-10, FP64, 64 standard-normal RHS.
    "lagtransform4096_2d_fp64": dict(
        plans=[("laguerre", 4096, {"scheme": "2d", "eta": 100.0})], eps=1e-10, precision="fp64", nrhs=64,
        dist="normal"),
}


def batch_workload(nplans: int = 1000, seed_offset: int = 3):
    """The many-plan batch: N log-uniform in [256, 8192], family uniform over
    {Chebyshev, Legendre, Jacobi(1/2,-1/2), Hermite functions}, 1..32 RHS."""
    g = rng(seed_offset)
    fams = ("chebyshev", "legendre", "jacobi", "hermite")
    out = []
    for _ in range(nplans):
        n = int(round(math.exp(g.uniform(math.log(256.0), math.log(8192.0)))))
        fam = fams[int(g.integers(0, len(fams)))]
        params = {"alpha": 0.5, "beta": -0.5} if fam == "jacobi" else {}
        nrhs = int(g.integers(1, 33))
        out.append((fam, n, params, nrhs))
    return out


def draw(dist: str, n: int, nrhs: int, *offsets: int) -> np.ndarray:
    """Dispatch on the distribution name used in WORKLOADS."""
    if dist == "uniform_pm1":
        return uniform_pm1(n, nrhs, *offsets)
    if dist == "uniform_01":
        return uniform_01(n, nrhs, *offsets)
    if dist == "normal":
        return normal(n, nrhs, *offsets)
    if dist == "complex_normal":
        return complex_normal(n, nrhs, *offsets)
    raise ValueError(f"unknown distribution {dist!r}")
