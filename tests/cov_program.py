"""The covariance program of Sec. 5.1 as a harness program: column means, centring, the
upper-triangular product C = X^T X / (n - 1) with each device's use of X narrowed to the columns
its rows need (absolute sections) and its definition to the upper trapezoid of its rows, then the
symmetric copy with the transposed use narrowed to one block per device and the definition to the
lower trapezoid.  Row blocks of C split evenly (the default partition) or balanced by the area of
the upper triangle (a manual partition, as in Listing 1).  With `correlation`, the centred columns
are scaled to unit norm before the product, which is then the correlation matrix."""

from paper_1809_05657_gb300.partitions import even_rows, triangle_balanced_rows as balanced_rows


def cov_prog(n, m, P, dtype="double", balanced=False, correlation=False):
    rows = balanced_rows(m, P) if balanced else even_rows(m, P)
    prog = [("create", "X", dtype, (n, m)), ("create", "M", dtype, (1, m)),
            ("create", "Xc", dtype, (n, m)), ("create", "C", dtype, (m, m)),
            ("part", "DX", 0, (n, m), (0, 0), (n, m), P),   # samples split by rows
            ("part", "PM", 1, (1, m), (0, 0), (1, m), P),   # means split by columns
            ("manual", "PC", (m, m), [((rows[p], 0), (rows[p + 1], m)) for p in range(P)]),
            ("write", "X", "DX"),
            ("apply", "colmean", "PM", ["X", "M"]),
            ("apply", "center", "DX", ["X", "M", "Xc"])]
    if correlation:  # scale the centred columns to unit norm: the product is then the correlation
        prog += [("create", "S", dtype, (1, m)), ("create", "Xs", dtype, (n, m)),
                 ("apply", "colnorm", "PM", ["Xc", "S"]),
                 ("apply", "colscale", "DX", ["Xc", "S", "Xs"])]
    src = "Xs" if correlation else "Xc"
    for p in range(P):
        r0, r1 = rows[p], rows[p + 1]
        prog.append(("abs_use", "syrk", "PC", src, p, (0, r0), (n, m)))
        prog.append(("trap_def", "syrk", "PC", "C", p, (r0, r0, r0, m - 1, r1 - 1, r1 - 1, r1 - 1, m - 1)))
        prog.append(("abs_use", "symmetrize", "PC", "C", p, (0, r0), (r1, r1)))
        t = max(r0, 1)
        if t < r1:
            prog.append(("trap_def", "symmetrize", "PC", "C", p, (t, 0, t, t - 1, r1 - 1, 0, r1 - 1, r1 - 2)))
        else:  # a device whose only row is row 0 defines nothing in the symmetric copy
            prog.append(("abs_def", "symmetrize", "PC", "C", p, (0, 0), (0, 0)))
    prog += [("apply", "syrk", "PC", [src, "C"], (1.0 if correlation else 1.0 / (n - 1),)),
             ("apply", "symmetrize", "PC", ["C"])]
    return prog, rows
