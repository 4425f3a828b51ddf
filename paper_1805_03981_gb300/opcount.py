"""Algorithmic operation and byte counts of the kernels, per element.

Flops count what the formulation requires: a 1D contraction producing one
value from m inputs costs 2m flops (m multiply-adds), point-wise operations
are counted one by one.  Bytes count compulsory device-memory traffic: each
state vector and geometry array read or written once per launch; face values
of neighbours are assumed to come from cache (the element's own read brings
them in), as the paper's measurements show for its CPU loops (Sec. 4.4).

Also here: the paper's own per-element operation-count model (Sec. 4.1,
C_tensorial and Table "kernel-calls"), used for comparison only.
"""


def contraction(outputs, m):
    return 2 * m * outputs


def eo_line(m):
    """Flops of one m-point line of a square centrosymmetric or
    skew-centrosymmetric contraction (V, V^-1, D) in the even-odd form the
    kernels use for m >= 5 (h = m // 2): h sums and h differences, two h x h
    products, h more multiply-adds with the middle value and the middle row
    for odd m, and h sums and h differences to combine; 2 m^2 below m = 5."""
    if m < 5:
        return 2 * m * m
    h = m // 2
    f = 2 * h + 4 * h * h + 2 * h
    if m % 2:
        f += 2 * h + 2 * h + 2
    return f


def sq_contraction(outputs, m):
    """A square V, V^-1 or D contraction producing `outputs` values along
    m-point lines (the even-odd count where the kernels use it)."""
    return outputs // m * eo_line(m)


def operator_flops(n, curved=True, nonwall_frac=1.0, basis="gl", affine=False):
    """R = -M^-1 K U on one element: basis changes, cell terms, faces, M^-1.
    basis "g": the state is held at the Gauss points (no basis changes; a
    neighbour trace is one l(+-1) contraction of the neighbour's line).
    affine (with basis "g"): constant metric; per direction one contraction
    of w sum_i adj_{d i} v_i and one of w p, distributed with adj_{d i}."""
    N3, N2 = n ** 3, n ** 2
    if basis == "g" and affine:
        f = 3 * N3 * (7 + 2 + 6) + 6 * contraction(N3, n) + 4 * N3
        f += 6 * N2 * (4 * 2 * n + 5 + 5 + 2 + 4 + 4 + 3 + 4 * 2 * n + 5)
        f += nonwall_frac * 6 * 4 * contraction(N2, n)
        f += 6 * N3
        return f
    if basis == "g":
        f = 3 * N3 * (5 + 3) + 12 * contraction(N3, n) + 2 * 4 * N3
        f += 6 * N2 * (4 * 2 * n + 5 + 5 + 2 + 4 + 4 + 3 + 4 * 2 * n)
        f += nonwall_frac * 6 * 4 * contraction(N2, n)
        f += 4 * N3
        return f
    f = 0
    f += 12 * sq_contraction(N3, n)         # GL -> G, 4 fields x 3 directions
    f += 3 * N3 * (5 + 3)                   # contravariant fluxes per direction
    f += 12 * contraction(N3, n)            # test-gradient (transposed derivative)
    f += 2 * 4 * N3                         # accumulation over the 3 directions
    face_pt = 4 * 2 * n + 5 + 5 + 2 + 4 + 4 + 3 + 4 * 2 * n
    f += 6 * N2 * face_pt                   # traces, flux, lifting
    f += nonwall_frac * 6 * 4 * 2 * sq_contraction(N2, n)   # neighbour GL face nodes -> Gauss
    f += 4 * N3                             # diagonal inverse mass
    f += 12 * sq_contraction(N3, n)         # G -> GL
    return f


EPILOGUE_FLOPS = {"operator": 0, "lsrk_stage": 5, "ader_update": 1}


def tck_levels(n, red):
    """(m, number of derivative evaluations at m, projections from m) for
    the Taylor terms j = 1..n (k + 1 = n), reduction every `red` steps."""
    seq = []
    m = n
    for j in range(1, n + 1):
        if m <= 0:
            break
        seq.append(m)
        if red and j % red == 0:
            m -= red
    return seq


def tck_flops(n, red=2, basis="gl", affine=False):
    N3 = n ** 3
    f = 0 if basis == "g" else 12 * sq_contraction(N3, n) + 12 * sq_contraction(N3, n)   # GL -> G, G -> GL
    deriv_contr, deriv_pt = (6, 36) if affine else (12, 36)
    f += 2 * 4 * N3                                          # first Taylor term
    m = n
    levels = [n]
    for j in range(1, n + 1):
        if m <= 0:
            break
        if m > 1:
            m3 = m ** 3
            f += deriv_contr * sq_contraction(m3, m) + deriv_pt * m3   # derivatives + chain rule
        if red and j % red == 0:
            if m - red < 1:
                break
            r = m - red
            f += 4 * (contraction(r * m * m, m) + contraction(r * r * m, m) + contraction(r ** 3, m))
            m = r
            levels.append(m)
        f += 2 * 4 * m ** 3                                  # accumulate the term
    for a, b in zip(levels[1:], levels[:-1]):                # fold small -> big
        f += 4 * (contraction(b * a * a, a) + contraction(b * b * a, a) + contraction(b ** 3, a))
        f += 4 * b ** 3
    return f


def tck_flops_alg1(n, affine=False):
    """The predictor without the basis change (Sec. 3.2, Alg. 1): per
    derivative, GL -> G interpolation (12 contractions), the collocation
    derivative and chain rule at the Gauss points, the w det J weights, the
    integration against the GL functions (12), and the inverse GL mass matrix
    V^-1 diag V^-T (24 and a division per point); no degree reduction.
    Once per element: w det J from the inverse Jacobian (about 30 per point)."""
    N3 = n ** 3
    deriv_contr, deriv_pt = (6, 36) if affine else (12, 36)
    per = (12 * contraction(N3, n) + deriv_contr * contraction(N3, n) + deriv_pt * N3 + 4 * N3
           + 12 * contraction(N3, n) + 24 * contraction(N3, n) + 4 * N3 + 2 * 4 * N3)
    return 30 * N3 + 4 * N3 + n * per


def geometry_reals(n, curved=True):
    """Per-element geometry values read by the operator: 9 metric + 2 mass
    diagonal per cell point, 6 per face point."""
    return 11 * n ** 3 + 36 * n ** 2


def tck_geometry_reals(n, red=2):
    """Predictor geometry values read per element: the Gauss sets visited."""
    lv = [n] if red == 0 else [m for m in range(n, 1, -red)]
    return 11 * sum(m ** 3 for m in lv)


AFF_OP, AFF_TCK = 48, 16   # compact per-element values of affine elements


def bytes_per_element(kind, n, rsize, red=2, first_stage=False, affine=False):
    vec = 4 * n ** 3 * rsize
    conn = 6 * (4 + 1 + 1)
    geo = (AFF_OP if affine else geometry_reals(n)) * rsize
    if kind == "operator":
        return 2 * vec + geo + conn
    if kind == "lsrk_stage":
        return (3 if first_stage else 4) * vec + geo + conn
    if kind == "ader_update":
        return 3 * vec + geo + conn
    if kind == "tck":
        return 2 * vec + (AFF_TCK if affine else tck_geometry_reals(n, red)) * rsize
    if kind == "other":
        return 2 * vec
    raise ValueError(kind)


def flops_per_element(kind, n, red=2, nonwall_frac=1.0, basis="gl", affine=False):
    if kind == "tck":
        return tck_flops(n, red, basis, affine)
    if kind == "other":                       # change of basis of a whole state
        return 12 * sq_contraction(n ** 3, n)
    return (operator_flops(n, nonwall_frac=nonwall_frac, basis=basis, affine=affine and basis == "g")
            + EPILOGUE_FLOPS[kind] * 4 * n ** 3)


# --- the paper's model (Sec. 4.1), for comparison --------------------------
def c_tensorial(k, delta):
    """Operations of one tensor-product kernel with even-odd decomposition:
    (2 (k+1)/2 * 2 + (k+1) + 2 floor((k-1)(k+1)/2)) (k+1)^(delta-1)."""
    return (2 * ((k + 1) / 2) * 2 + (k + 1) + 2 * (((k - 1) * (k + 1)) // 2)) * (k + 1) ** (delta - 1)


def paper_kernel_calls(k, d=3):
    """(cell, face) tensor-kernel calls of M^-1, K and TCK (Table kernel-calls)."""
    return {"mass": (2 * d, 0), "stiffness": (d * d + 4 * d, 4 * (d * d - d)),
            "tck": (2 * d + d * (k - 1), 0)}


def paper_scheme_ops(k, d=3, stages=5):
    """Operations per element and step of the paper's model (Sec. 4.1):
    C_RK = s (C_M + C_K) and C_ADER = 2 C_M + C_K + C_TCK, where a cell
    kernel call costs C_tensorial(d) and a face kernel call C_tensorial(d-1)
    (Table kernel-calls)."""
    C, F = c_tensorial(k, d), c_tensorial(k, d - 1)
    calls = paper_kernel_calls(k, d)
    cost = {name: cf[0] * C + cf[1] * F for name, cf in calls.items()}
    return {"rk": stages * (cost["mass"] + cost["stiffness"]),
            "ader": 2 * cost["mass"] + cost["stiffness"] + cost["tck"], **cost}
