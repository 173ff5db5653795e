"""Algorithmic FLOP and byte counts of the kernels, for roofline reporting.

Counts follow the formulas the kernels evaluate (an FMA is 2 flops; an add,
multiply, divide, square root, log, sine/cosine or atan2 is 1), with the
triangular structure of the factors taken into account.  Per-launch totals
use the same chunking as the library's plan (leaf chunks of ``leaf`` steps,
upper levels of ``radix`` items, or the adaptive 4 / 32 choice for radix 0).
Upper levels count the work-efficient number of combines (c - 1 per chunk of
c items); the warp-scanned chunks do more.
"""
import math


def tria(R, C, nref=None):
    """Householder LQ of an R x C block (Tria, Sec. 2.2)."""
    nref = R if nref is None else nref
    f = 0
    for i in range(nref):
        w = C - i
        f += 2 * w + 6                      # norm, sqrt, v0, tau
        f += (R - 1 - i) * (4 * w + 1)      # dot + scale + update per row
    return f


def tri_mm(M, NX):
    """M x NX times a lower NX x NX factor."""
    return M * NX * (NX + 1)


def kf_step(nx, ny):
    W = nx + ny
    return (2 * nx * nx + nx + tri_mm(nx, nx) + tria(nx, 2 * nx) + tri_mm(ny, nx)
            + tria(W, W) + ny * (2 * nx + 2) + ny * ny + 4 * ny + 3 + nx * 2 * ny)


def filter_element(nx, ny):
    W = nx + ny
    return (tri_mm(ny, nx) + tria(W, W) + 2 * ny * (2 * nx + 2) + 2 * ny * ny
            + 2 * nx * ny + 2 * ny * nx * nx + nx * ny * ny + 2 * nx * nx * ny + 2 * nx * ny)


def xi_blocks(nx):
    """M = U_i^T Z_j (U_i lower), Xi_11 = Tria([M, I]) and the gain
    G = Z_j M^T Xi_11^{-T} Xi_11^{-1} (product, two triangular solves)."""
    tri = nx * nx * (nx + 1)            # a triangular solve / product, 2 flops per FMA
    return tri + tria(nx, 2 * nx) + 2 * nx ** 3 + 2 * tri


def filter_combine(nx):
    tri = nx * nx * (nx + 1)
    ab = tri + 4 * nx ** 3 + 2 * (nx * (nx + 1) + nx * nx) + 2 * nx       # I - U G^T, A, b
    eta = 2 * (3 * nx * nx + nx * (nx + 1)) + 3 * nx
    u = 2 * nx ** 3 + tri + tria(nx, 2 * nx)                              # A_j U_i Xi_11^{-T}
    z = tria(nx, 2 * nx) + tri + 2 * nx ** 3 + tria(nx, 2 * nx)            # L, W, A_i^T W
    return xi_blocks(nx) + ab + eta + u + z


def filter_apply(nx):
    tri = nx * nx * (nx + 1)
    b = 2 * (nx * (nx + 1) + 2 * nx * nx) + 3 * nx
    return xi_blocks(nx) + b + 2 * nx ** 3 + tri + tria(nx, 2 * nx)


def smoother_element(nx):
    return (tri_mm(nx, nx) + tria(2 * nx, 2 * nx) + nx ** 3 + 4 * nx * nx + 2 * nx)


def smoother_combine(nx):
    return 2 * nx ** 3 + 2 * nx * nx + nx + tri_mm(nx, nx) + tria(nx, 2 * nx)


def smoother_apply(nx):
    return 2 * nx * nx + nx + tri_mm(nx, nx) + tria(nx, 2 * nx)


# The mean-only smoother of the refinement passes (E_k read back, no Tria):
# g = m^f - E (F m^f + c); E_ij = E_i E_j, g_ij = E_i g_j + g_i; g <- E g + g_i.
def smoother_element_g(nx):
    return 4 * nx * nx + 2 * nx


def smoother_combine_g(nx):
    return 2 * nx ** 3 + 2 * nx * nx + nx


def smoother_apply_g(nx):
    return 2 * nx * nx + nx


# The mean-only upper filter levels of the refinement passes: b_ij, eta_ij of
# Table 3 from the factors the full pass stored -- three triangular products
# with U_i, two with Z_j, three full ones (A_j (I - U_i G^T), G, A_i^T) and
# five vector sums.  The library takes that form, in FP32, for levels of at
# most CS3_MAX_CHUNKS chunks (the three-role chunk levels and the top) when a
# batch has at most FMEANS_MAX_SEQS sequences and the state at least
# FMEANS_MIN_NX entries.
CS3_MAX_CHUNKS = 512
FMEANS_MAX_SEQS = 64
FMEANS_MIN_NX = 3


def filter_combine_means(nx):
    return 5 * nx * (nx + 1) + 6 * nx * nx + 5 * nx


# CT cubature SLR: per sigma point the transition difference costs two turn
# coefficient evaluations (sincos x2, series or divide) and ~24 flops; a
# bearing difference costs ~8 flops + atan2 per sensor.
CT_F_DELTA = 2 * 12 + 24
CT_H_DELTA = 2 * (9 + 1)


def slr_cubature_ct(nx=5, ny=2):
    tr = (20 + 2 * nx * CT_F_DELTA + nx * nx * 4 + nx * nx * nx + 2 * nx * nx
          + nx * (2 * nx) + tria(nx, 2 * nx))
    ob = (2 * 10 + 2 * nx * CT_H_DELTA + ny * nx * 4 + ny * nx * nx + 2 * ny * nx
          + ny * (nx + ny) + tria(ny, ny + nx) + 2 * 4)
    return tr + ob


def slr_taylor_ct(nx=5, ny=2):
    return 20 + 40 + 2 * nx * nx + 2 * (10 + 10) + 2 * ny * nx + 8


def _chunks(counts, size):
    """Chunk sizes of one level and the item counts of the next."""
    sizes, nxt = [], []
    for c in counts:
        nch = (c + size - 1) // size
        sizes += [min(size, c - j * size) for j in range(nch)]
        nxt.append(nch)
    return sizes, nxt


# Adaptive plans (radix 0) fold a level of more items than this 4 per thread
# and scan smaller levels in chunks of 32 (one warp per chunk).
FOLD_ABOVE_ITEMS = 160000


def default_leaf(steps, sm_count=152):
    """Leaf chunk the library picks when none is given: 3 while the leaf
    chunks fit one wave of 256 threads per SM, else 4."""
    return 3 if steps <= 3 * 256 * sm_count else 4


def _levels(counts0, leaf, radix):
    levels = []
    counts = list(counts0)
    size = leaf
    while True:
        sizes, nxt = _chunks(counts, size)
        levels.append(sizes)
        counts = nxt
        if radix > 1:
            size = radix
        else:
            size = 32 if sum(counts) <= FOLD_ABOVE_ITEMS else 4
        if all(c == 1 for c in counts):
            return levels


def ipls_kernel_flops(lengths, nx=5, ny=2, leaf=None, radix=0, linearization="cubature",
                      refine=0):
    """Algorithmic flops per launch of each kernel family for one IPLS
    iteration over sequences of the given lengths; with `refine` passes the
    filter scan runs 1 + refine times per iteration (its latency-bound upper
    levels mean-only in the refinement passes of a batch of at most
    FMEANS_MAX_SEQS sequences; FP32) and the smoother scan once in full and
    `refine` times mean-only (flops per launch then the average over its
    passes).  Returns {family: (flops per launch, launches per iteration)}."""
    out = {}
    nsteps = sum(lengths)
    leaf = default_leaf(nsteps) if leaf is None else leaf
    slr = slr_cubature_ct(nx, ny) if linearization == "cubature" else slr_taylor_ct(nx, ny)
    out["ct_slr"] = (nsteps * slr, 1)
    fl = _levels(lengths, leaf, radix)
    sl = _levels([n + 1 for n in lengths], leaf, radix)
    fe, fc, fa = filter_element(nx, ny), filter_combine(nx), filter_apply(nx)
    if len(fl) > 1:
        out["filter_leaf_up"] = (sum(c * fe + (c - 1) * fc for c in fl[0]), 1)
    ups = [sum((c - 1) * fc for c in lv) for lv in fl[1:]]
    downs = [sum((c - 1) * fa for c in lv) for lv in fl[1:]]
    if ups:
        out["filter_up"] = (sum(ups) / len(ups), len(ups))
        out["filter_down"] = (sum(downs) / len(downs), len(downs))
    out["filter_leaf_down"] = (nsteps * kf_step(nx, ny), 1)
    nel = nsteps + len(lengths)

    def smoother(se, sc, sa):
        sm = {}
        if len(sl) > 1:
            sm["smoother_leaf_up"] = (sum(c * se + (c - 1) * sc for c in sl[0])
                                      - len(lengths) * se, 1)
        ups = [sum((c - 1) * sc for c in lv) for lv in sl[1:]]
        downs = [sum((c - 1) * sa for c in lv) for lv in sl[1:]]
        if ups:
            sm["smoother_up"] = (sum(ups) / len(ups), len(ups))
            sm["smoother_down"] = (sum(downs) / len(downs), len(downs))
        sm["smoother_leaf_down"] = ((nel - len(lengths)) * (se + sa), 1)
        return sm
    full = smoother(smoother_element(nx), smoother_combine(nx), smoother_apply(nx))
    out.update(full)
    if refine:
        # each refinement pass: the filter scan again (its small upper levels
        # mean-only for few sequences), the smoother scan mean-only
        # (chunk-scan level shapes, the default ones)
        out = {k: (f, n * (1 + refine)) if k.startswith("filter") else (f, n)
               for k, (f, n) in out.items()}
        if ups and len(lengths) <= FMEANS_MAX_SEQS and nx >= FMEANS_MIN_NX:
            fm = filter_combine_means(nx)
            ups_r = [sum((c - 1) * (fm if len(lv) <= CS3_MAX_CHUNKS else fc) for c in lv)
                     for lv in fl[1:]]
            out["filter_up"] = ((sum(ups) + refine * sum(ups_r)) / (len(ups) * (1 + refine)),
                                len(ups) * (1 + refine))
        mean = smoother(smoother_element_g(nx), smoother_combine_g(nx), smoother_apply_g(nx))
        for k, (f, n) in full.items():
            fg, _ = mean[k]
            out[k] = ((f + refine * fg) / (1 + refine), n * (1 + refine))
    return out


def ipls_iteration_flops(lengths, **kw):
    return sum(f * n for f, n in ipls_kernel_flops(lengths, **kw).values())


def ipls_iteration_bytes(lengths, nx=5, ny=2, elem=4):
    """Algorithmic HBM bytes of one IPLS iteration with every phase's
    per-step inputs and outputs read / written once: y, the nominal
    trajectory (mean + packed lower factor) in and out."""
    tri = nx * (nx + 1) // 2
    nsteps = sum(lengths)
    rows = nsteps + len(lengths)
    return elem * (nsteps * ny + 2 * rows * (nx + tri))
