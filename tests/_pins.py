"""Independent checks used to pin the CPU oracle.

Each routine computes the local alignment score by a route other than the
Gotoh recurrences the oracle implements:

* ``brute_force``   -- enumerate every alignment of every pair of substrings
  and score it by the definition (sum of substitution scores minus, for each
  maximal run of k gap positions in one sequence, ``gap_open + k*gap_extend``).
* ``ungapped_best`` -- the best gap-free local alignment: Kadane's maximum
  sub-array sum along every diagonal of the substitution grid.
* ``linear_gap_sw`` -- Smith & Waterman (1981) with a linear gap penalty
  ``g`` per gap position, one-matrix recurrence.
* ``literal_gotoh`` -- Eqs. 1-3 with the paper's own Go/Ge symbols, used only
  to test how this library's (gap_open, gap_extend) convention maps onto them.
"""

import numpy as np


def brute_force(q, d, sm, gap_open, gap_extend):
    q = [int(x) for x in q]
    d = [int(x) for x in d]
    m, n = len(q), len(d)
    best = 0
    # depth-first walk over alignment paths; every prefix of a path is an
    # alignment of Q[a..i) with D[c..j).  last: 0 = match, 1 = gap in Q
    # (consumes D), 2 = gap in D (consumes Q), -1 = start.
    stack = []
    for a in range(m + 1):
        for c in range(n + 1):
            stack.append((a, c, -1, 0))
    while stack:
        i, j, last, s = stack.pop()
        if s > best:
            best = s
        if i < m and j < n:
            stack.append((i + 1, j + 1, 0, s + int(sm[q[i]][d[j]])))
        if j < n:
            cost = gap_extend if last == 1 else gap_open + gap_extend
            stack.append((i, j + 1, 1, s - cost))
        if i < m:
            cost = gap_extend if last == 2 else gap_open + gap_extend
            stack.append((i + 1, j, 2, s - cost))
    return best


def ungapped_best(q, d, sm):
    m, n = len(q), len(d)
    best = 0
    for off in range(-(m - 1), n):
        run = 0
        for i in range(m):
            j = i + off
            if 0 <= j < n:
                run = max(0, run + int(sm[int(q[i])][int(d[j])]))
                best = max(best, run)
    return best


def linear_gap_sw(q, d, sm, g):
    m, n = len(q), len(d)
    H = np.zeros((m + 1, n + 1), dtype=np.int64)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            H[i, j] = max(0, H[i - 1, j - 1] + int(sm[int(q[i - 1])][int(d[j - 1])]),
                          H[i - 1, j] - g, H[i, j - 1] - g)
    return int(H.max())


def literal_gotoh(q, d, sm, Go, Ge):
    """Eqs. 1-3 exactly as printed, with the paper's Go and Ge."""
    m, n = len(q), len(d)
    H = np.zeros((m + 1, n + 1), dtype=np.int64)
    E = np.zeros((m + 1, n + 1), dtype=np.int64)
    F = np.zeros((m + 1, n + 1), dtype=np.int64)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            E[i, j] = max(H[i, j - 1] - Go, E[i, j - 1] - Ge)
            F[i, j] = max(H[i - 1, j] - Go, F[i - 1, j] - Ge)
            H[i, j] = max(0, H[i - 1, j - 1] + int(sm[int(q[i - 1])][int(d[j - 1])]), E[i, j], F[i, j])
    return int(H.max())


def alignment_score(q, d, sm, gap_open, gap_extend, q_begin, t_begin, ops):
    """Score of an alignment given as operations (M: Q[i] with D[j]; I: Q[i]
    against a gap; D: D[j] against a gap) starting at (q_begin, t_begin): the
    substitution scores of the M pairs minus gap_open + k * gap_extend per
    maximal run of k I's or k D's.  Raises if the walk leaves a sequence."""
    i, j, total, prev = q_begin, t_begin, 0, None
    for op in ops:
        if op == "M":
            total += int(sm[int(q[i]), int(d[j])])
            i += 1
            j += 1
        elif op in "ID":
            total -= gap_extend + (gap_open if op != prev else 0)
            if op == "I":
                i += 1
            else:
                j += 1
        else:
            raise ValueError(op)
        if i > len(q) or j > len(d):
            raise ValueError("alignment runs past a sequence")
        prev = op
    return total, i, j

