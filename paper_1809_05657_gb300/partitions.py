"""Row splits for manual partitions (the `partition` clause of Listing 1, HDArrayPartitionManual).

even_rows: the default even split of the library's ROW partition (the first n mod P parts get one
extra row).  triangle_balanced_rows: row blocks of an m x m array whose work is the upper triangle
(m - i cells in row i), cut so that every block has the same number of cells -- the balanced
manual partition the paper uses for its triangular kernels (Sec. 5.1)."""

import math


def even_rows(m, P):
    return [p * (m // P) + min(p, m % P) for p in range(P + 1)]


def triangle_balanced_rows(m, P):
    """Boundaries r_0 = 0 < r_1 < ... < r_P = m with equal upper-triangle area per block."""
    total = m * (m + 1) / 2
    bounds = [0]
    for p in range(1, P):
        target = total * p / P
        # area of rows [0, r): r*m - r*(r-1)/2 = target, solved for r and rounded
        a, b, c = -0.5, m + 0.5, -target
        r = (-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)
        bounds.append(min(m - 1, max(bounds[-1] + 1, int(round(r)))))
    bounds.append(m)
    return bounds
