"""Seeded synthetic inputs for the triangular solve.

This module holds random-number generation only (no solver arithmetic); the
tests hand the same arrays to the CUDA path and to the CPU oracle.

Recipe (the paper's Section VI uses no public data set; every input here is
synthetic):
  * generator: ``numpy.random.default_rng(seed)`` (PCG64), FP64 on the host;
  * fill order: the full k x k array of A column-major, then the diagonal,
    then B column-major (k = m for side Left, n for side Right);
  * off-diagonal entries of A: U(-1, 1) / k;  diagonal: U[1, 2);
  * B: standard normal;
  * the triangle of A that op(A) does not reference is set to zero (or NaN
    when ``poison=True``; with a unit diagonal the diagonal is then NaN too,
    since it must not be read).
With the diagonal >= 1 and each row's off-diagonal absolute sum < 1, A is
strictly diagonally dominant, hence well conditioned.

Device recipe (``make_problem_device``, for sizes whose host generation would
be slow, e.g. k = 32768): the same distributions drawn on the GPU by a torch
generator seeded with ``seed`` (a different stream of numbers than the host
recipe), the unreferenced triangle zero.

Cholesky recipe (``make_spd``, ``make_spd_device``): a symmetric A with the
triangle recipe's entries, off-diagonal (U(-1, 1) + U(-1, 1)^T) / (2k) and
diagonal U[1, 2), so every row's off-diagonal absolute sum is below the
diagonal: symmetric, strictly diagonally dominant with a positive diagonal,
hence positive definite and well conditioned; both triangles are stored.

Batched recipe: ``SeedSequence(seed).spawn(count)``; per instance
m = round(exp(U(ln 16, ln 512))), n = integers(1, 257), side and uplo uniform
over {0, 1}, trans = NoTrans, diag = NonUnit, alpha = 1.
"""
import numpy as np

LEFT, RIGHT = 0, 1
LOWER, UPPER = 0, 1
NOTRANS, TRANS = 0, 1
NONUNIT, UNIT = 0, 1


def make_triangle(k, uplo, diag, rng, poison=False):
    off = rng.uniform(-1.0, 1.0, size=k * k).reshape((k, k), order="F") / max(k, 1)
    d = rng.uniform(1.0, 2.0, size=k)
    A = np.asfortranarray(off)
    A[np.diag_indices(k)] = d
    fill = np.nan if poison else 0.0
    if uplo == LOWER:
        A[np.triu_indices(k, 1)] = fill
    else:
        A[np.tril_indices(k, -1)] = fill
    if poison and diag == UNIT:
        A[np.diag_indices(k)] = np.nan
    return A


def make_problem(side, uplo, trans, diag, m, n, seed, poison=False):
    """Return (A, B): A k x k column-major FP64, B m x n column-major FP64."""
    rng = np.random.default_rng(seed)
    k = m if side == LEFT else n
    A = make_triangle(k, uplo, diag, rng, poison)
    B = np.asfortranarray(rng.standard_normal(m * n).reshape((m, n), order="F"))
    return A, B


def batch_shapes(count, seed):
    """Per-instance (side, uplo, m, n, seed) of the uneven batch."""
    out = []
    for child in np.random.SeedSequence(seed).spawn(count):
        rng = np.random.default_rng(child)
        m = int(round(float(np.exp(rng.uniform(np.log(16.0), np.log(512.0))))))
        n = int(rng.integers(1, 257))
        side = int(rng.integers(0, 2))
        uplo = int(rng.integers(0, 2))
        out.append((side, uplo, m, n, int(rng.integers(0, 2**63 - 1))))
    return out


def make_batch(count, seed):
    """List of dicts with keys side, uplo, trans, diag, m, n, alpha, A, B."""
    items = []
    for side, uplo, m, n, s in batch_shapes(count, seed):
        A, B = make_problem(side, uplo, NOTRANS, NONUNIT, m, n, s)
        items.append(dict(side=side, uplo=uplo, trans=NOTRANS, diag=NONUNIT,
                          m=m, n=n, alpha=1.0, A=A, B=B))
    return items


def make_problem_device(side, uplo, trans, diag, m, n, seed):
    """(A, B) as column-major torch FP64 CUDA tensors with the distributions
    of ``make_problem`` (different random numbers), generated on the GPU."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    k = m if side == LEFT else n
    # column-major k x k: the transpose of a row-major buffer
    A = torch.empty((k, k), dtype=torch.float64, device="cuda").t()
    A.uniform_(-1.0, 1.0, generator=g).div_(max(k, 1))
    A.diagonal().uniform_(1.0, 2.0, generator=g)
    if uplo == LOWER:
        A.copy_(torch.tril(A))
    else:
        A.copy_(torch.triu(A))
    B = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
    B.normal_(generator=g)
    return A, B


def make_spd(k, seed):
    """Symmetric positive definite k x k FP64 (column-major), both triangles."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(-1.0, 1.0, size=k * k).reshape((k, k), order="F") / max(k, 1)
    A = np.asfortranarray((off + off.T) / 2.0)
    A[np.diag_indices(k)] = rng.uniform(1.0, 2.0, size=k)
    return A


def make_spd_device(k, seed):
    """As make_spd, drawn on the GPU (torch generator; different numbers)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    A = torch.empty((k, k), dtype=torch.float64, device="cuda").t()
    A.uniform_(-1.0, 1.0, generator=g).div_(max(k, 1))
    A.add_(A.t().clone()).mul_(0.5)
    A.diagonal().uniform_(1.0, 2.0, generator=g)
    return A
