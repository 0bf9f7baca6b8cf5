"""The paper's computation models (Section V) -- TEST INFRASTRUCTURE ONLY.

Plain restatement of the task structure and cost formulas of the recursive
(Section V-A), iterative (Section V-B) and blocked (Section V-C) models, used
to check the library's schedules and its analytic planner.

Notation as in the paper: iteration i, refinement level r(i) = 2^i (Eq. 1);
TS(i) is the time of one diagonal (TS) task at iteration i, gemm(j) the time
of one GEMM task of recursion level j, gemm(i, j) the j-th GEMM of the
iterative model, gemm(i) one off-diagonal block of the blocked model.
"""


def refinement_level(i):
    """Eq. (1): r(i) = 2^i."""
    return 2 ** i


def refine_further(ts_i, ts_next):
    """Section V-A condition: refine from iteration i to i+1 only if
    2 * TS(i+1) < TS(i) (strict)."""
    return 2 * ts_next < ts_i


def recursive_tasks(i, n):
    """Recursive model at iteration i for order n (a power of two):
    r(i) TS tasks of order n / 2^i, and at each level j < i, r(j) GEMM tasks
    of size (n / 2^(j+1)) x (n / 2^(j+1))."""
    ts = [n // 2 ** i] * refinement_level(i)
    gemms = []
    for j in range(i):
        s = n // 2 ** (j + 1)
        gemms += [(s, s)] * refinement_level(j)
    return ts, gemms


def recursive_comp(i, TS, gemm):
    """Comp(i) = r(i) TS(i) + sum_{j=0}^{i-1} r(j) gemm(j)."""
    return refinement_level(i) * TS(i) + sum(refinement_level(j) * gemm(j) for j in range(i))


def iterative_tasks(i):
    """Iterative model: r(i) TS tasks and GEMMs gemm(i, j), j = 0..r(i)-2."""
    r = refinement_level(i)
    return r, r - 1


def iterative_comp(i, TS, gemm_ij):
    """Comp(i) = r(i) TS(i) + sum_{j=0}^{r(i)-2} gemm(i, j)."""
    r = refinement_level(i)
    return r * TS(i) + sum(gemm_ij(i, j) for j in range(r - 1))


def blocked_rounds(i):
    """Blocked model: r(i) - 1 rounds of r(i)/2 blocks each."""
    r = refinement_level(i)
    return r - 1, r // 2


def blocked_blocks(i):
    """Total off-diagonal GEMM blocks: (r(i) - 1) * r(i) / 2."""
    rounds, per = blocked_rounds(i)
    return rounds * per


def blocked_comp(i, TS, gemm):
    """Comp(i) = r(i) TS(i) + ((r(i) - 1) r(i) / 2) gemm(i)."""
    return refinement_level(i) * TS(i) + blocked_blocks(i) * gemm(i)
