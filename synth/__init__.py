"""Seeded synthetic inputs shaped like the paper's workloads.

Shared by the tests, the oracle checks and the benchmark; holds none of the
method's arithmetic (no split, no projection, no factorisation beyond the
Haar-matrix recipe that builds test matrices).

Every generator takes an explicit seed and draws from
``numpy.random.default_rng(seed)`` (PCG64) in a fixed, documented order, so
the CPU oracle and the GPU path always see the same bytes.

Recipes
-------
haar(n, k, rng)            n x k matrix with orthonormal columns, Haar
                           distributed: QR of an n x k N(0,1) matrix with the
                           signs of diag(R) folded in (Mezzadri, 2007).
omega_f16(n, k, seed)      N(0,1) drawn in FP32, rounded RN-even to FP16
                           (Sec. 3.3 generates the Gaussian in FP32 and rounds).
planted_svd(m, n, sigma, seed)
                           A = U diag(sigma) V^T, U then V Haar (the RSVD
                           accuracy test matrices of Sec. 5.1 with the planted
                           spectrum stated by the caller).
uniform(m, n, seed, lo, hi) i.i.d. U[lo, hi) FP32 (the SHGEMM accuracy inputs
                           of Sec. 4.4.1).
tucker(dims, core, seed, noise_std)
                           core N(0,1), factors Haar, plus i.i.d. N(0,
                           noise_std^2) noise; the RP-HOSVD test tensor.
hosvd_omegas(dims, J, seed) one FP16 Gaussian per mode of a 3-way tensor.
batch_specs(count, seed)   (m, n, rate, rank, seed) of a batch of uneven
                           matrices; batch_matrix(spec) builds one of them.
sketch_basis(n, r, seed), sketch_matrix(V0, m, sigma, theta_max, noise_rel, seed)
                           matrices U diag(sigma) (V0 cos T + W sin T)^T + E of
                           the learned-sketch family.
cauchy_family(n, seed)     Cauchy matrix after one orthogonal-iteration step,
                           entries beyond the FP16 range (SHGEMM-TF32 inputs).
"""
from __future__ import annotations

import numpy as np


def haar(n: int, k: int, rng: np.random.Generator) -> np.ndarray:
    G = rng.standard_normal((n, k))
    Q, R = np.linalg.qr(G, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def omega_f16(n: int, k: int, seed: int) -> np.ndarray:
    """n x k float16 array, N(0,1) in FP32 then RN-even to FP16 (seed)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, k), dtype=np.float32)
    return g.astype(np.float16)


def planted_svd(m: int, n: int, sigma: np.ndarray, seed: int) -> np.ndarray:
    """FP32 m x n matrix U diag(sigma) V^T; U (m x r) then V (n x r) from seed."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    U = haar(m, r, rng)
    V = haar(n, r, rng)
    return ((U * np.asarray(sigma, dtype=np.float64)) @ V.T).astype(np.float32)


def sigma_exp(count: int, rate: float) -> np.ndarray:
    """sigma_i = 2^(-i / rate), i = 1..count (1-based as in Sec. 2.1)."""
    i = np.arange(1, count + 1, dtype=np.float64)
    return 2.0 ** (-i / rate)


def uniform(m: int, n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(m, n)).astype(np.float32)


def rsvd_planted(m: int = 1024, n: int = 1024, rate: float = 8.0, seed_a: int = 0,
                 seed_omega: int = 1, k: int = 64):
    """The randomized-SVD accuracy workload: A = U diag(2^(-i/rate)) V^T with
    U, V Haar from ``seed_a`` (full rank min(m, n)), Omega n x k from
    ``seed_omega``."""
    r = min(m, n)
    A = planted_svd(m, n, sigma_exp(r, rate), seed_a)
    return A, omega_f16(n, k, seed_omega)


def tucker(dims, core_dims, seed: int, noise_std: float = 1e-4):
    """Tucker tensor: core N(0,1) (drawn first), then one Haar factor per mode
    in mode order, then the noise.  Returns (A float32, core, factors)."""
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(core_dims))
    facs = [haar(I, J, rng) for I, J in zip(dims, core_dims)]
    T = core
    for i, F in enumerate(facs):
        T = np.moveaxis(np.tensordot(T, F, axes=([i], [1])), -1, i)
    if noise_std:
        T = T + noise_std * rng.standard_normal(T.shape)
    return T.astype(np.float32), core, facs


def hosvd_omegas(dims, J, seed: int):
    """One FP16 Gaussian per mode: (prod_{j != i} I_j) x J_i, drawn in mode order."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(len(dims)):
        rows = int(np.prod([d for j, d in enumerate(dims) if j != i]))
        out.append(rng.standard_normal((rows, J[i]), dtype=np.float32).astype(np.float16))
    return out


def batch_specs(count: int, seed: int, m_range=(256, 4096), n_range=(256, 2048),
                r_range=(8, 64), ranks=(16, 32, 64, 128)):
    """Shapes of a batch of uneven matrices: m, n uniform integers in the
    (inclusive) ranges, decay rate r uniform in r_range, target rank uniform
    over ``ranks`` and clipped so that rank + 16 <= min(m, n)."""
    rng = np.random.default_rng(seed)
    m = rng.integers(m_range[0], m_range[1] + 1, size=count)
    n = rng.integers(n_range[0], n_range[1] + 1, size=count)
    r = rng.uniform(r_range[0], r_range[1], size=count)
    rank = rng.choice(np.asarray(ranks), size=count)
    rank = np.minimum(rank, np.minimum(m, n) - 16)
    return [dict(m=int(a), n=int(b), rate=float(c), rank=int(d), seed=int(seed * 100003 + i))
            for i, (a, b, c, d) in enumerate(zip(m, n, r, rank))]


def batch_matrix(spec) -> np.ndarray:
    """FP32 m x n matrix with sigma_i = 2^(-i/rate) from spec['seed']."""
    r = min(spec["m"], spec["n"])
    return planted_svd(spec["m"], spec["n"], sigma_exp(r, spec["rate"]), spec["seed"])


def sketch_basis(n: int, r: int, seed: int) -> np.ndarray:
    """The fixed orthonormal basis V0 (n x r) of the learned-sketch family."""
    return haar(n, r, np.random.default_rng(seed))


def sketch_matrix(V0: np.ndarray, m: int, sigma: np.ndarray, theta_max: float,
                  noise_rel: float, seed: int) -> np.ndarray:
    """A = U diag(sigma) (V0 cos(Theta) + W sin(Theta))^T + E.

    U is Haar (m x r); W is a Haar basis of the orthogonal complement of V0
    (Haar n x r matrix projected and re-orthonormalised); Theta = diag(theta_j)
    with theta_j ~ U[0, theta_max]; E is Gaussian scaled so that
    ||E||_F = noise_rel * ||signal||_F.  Draw order: U, W, theta, E.
    """
    n, r = V0.shape
    rng = np.random.default_rng(seed)
    U = haar(m, r, rng)
    W = rng.standard_normal((n, r))
    W = W - V0 @ (V0.T @ W)
    W, Rw = np.linalg.qr(W)
    W = W * np.sign(np.diag(Rw))
    th = rng.uniform(0.0, theta_max, size=r)
    V = V0 * np.cos(th) + W * np.sin(th)
    S = (U * sigma) @ V.T
    E = rng.standard_normal((m, n))
    E *= noise_rel * np.linalg.norm(S) / np.linalg.norm(E)
    return (S + E).astype(np.float32)


def cauchy_family(n: int, seed: int, gamma: float = 1e-3, spread: float = 1e-3) -> np.ndarray:
    """Stand-in for the Cauchy matrices of the randomized-SVD experiments:
    C_ij = 1 / (|x_i - y_j| + gamma) with x, y uniform in (-spread, spread)
    (x drawn first), followed by one step of the orthogonal iteration applied
    to the matrix, A = (C C^T) C, formed in float64 and rounded to FP32.  Its
    entries (about n^2 10^9) exceed the FP16 range, the case SHGEMM-TF32 is
    for."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-spread, spread, size=n)
    y = rng.uniform(-spread, spread, size=n)
    C = 1.0 / (np.abs(x[:, None] - y[None, :]) + gamma)
    return ((C @ C.T) @ C).astype(np.float32)
