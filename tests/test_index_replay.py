"""CPU replays of the CUDA kernels' index arithmetic (no GPU, no library
call): for every shape the kernels are launched with, each shared-memory,
table and global index is checked against its buffer's extent, and each
pass that permutes data writes every element exactly once.  These are the
same expressions as the kernels', restated in Python, run before any new
kernel shape reaches the GPU; the bounds-checked build
(tests/test_gpu_bounds_check.py) checks the same indices on the device.
"""
import itertools

import numpy as np
import pytest

# ---- warp-group FFT engine (csrc/solve32.cu) --------------------------------


def px(m):
    return m + (m >> 4)


def geo32(lg, rad):
    lr = rad.bit_length() - 1
    L = 1 << lg
    return dict(L=L, N=L // 2, G=L // rad, np=lg // lr, rem=lg % lr, buf=px(L) + 2)


def max_cta(rad, esz):
    return 512 if (rad == 16 and esz == 4) else 256


def supported(mx, rad, esz):
    lx, lr = (2 * mx).bit_length() - 1, rad.bit_length() - 1
    lt = max_cta(rad, esz).bit_length() - 1
    return lx >= lr and lx <= lr + lt


def stockham_passes(lg, rad):
    """(radix, NS) of the passes of one FFT of length 2^lg."""
    g = geo32(lg, rad)
    out, ns = [], 1
    for _ in range(g["np"]):
        out.append((rad, ns))
        ns *= rad
    if g["rem"]:
        out.append((1 << g["rem"], ns))
    return out


CASES32 = [(lg, rad, esz) for rad in (8, 16, 32) for esz in (4, 8) for lg in range(3, 14)
           if supported(1 << (lg - 1), rad, esz)]


@pytest.mark.parametrize("lg,rad,esz", CASES32)
def test_warp_group_fft_passes_stay_in_their_buffers(lg, rad, esz):
    g = geo32(lg, rad)
    L, G, buf = g["L"], g["G"], g["buf"]
    t = np.arange(G)
    for p, (R, NS) in enumerate(stockham_passes(lg, rad)):
        B = rad // R                       # butterflies per thread (remainder pass)
        j = (t[:, None] + np.arange(B)[None, :] * G).ravel()
        k = j & (NS - 1)
        r = np.arange(R)
        reads = j[:, None] + r[None, :] * (L // R)
        writes = (j - k)[:, None] * R + k[:, None] + r[None, :] * NS
        if p == 0:
            # the first pass reads the odd extension from the N stored values:
            # element m = t + r G is z_m (r < R/2), 0 (m = N) or -z_{L-m}
            H = R // 2
            m = t[:, None] + r[None, :] * G
            src = np.where(r[None, :] < H, m,
                           np.where(r[None, :] == H, g["N"] - t[:, None], (R - r[None, :]) * G - t[:, None]))
            assert src.min() >= 0 and src.max() <= g["N"]
            reads = src
        assert reads.min() >= 0 and reads.max() < L
        assert px(reads.max()) < buf
        # each pass writes every element of the length-L buffer exactly once
        assert np.array_equal(np.sort(writes.ravel()), np.arange(L))
        assert px(writes.max()) < buf


@pytest.mark.parametrize("mx,my,rad,esz", [(m, n, rad, esz) for rad in (8, 16, 32) for esz in (4, 8)
                                          for m, n in ((8, 8), (32, 64), (512, 1024), (1024, 512),
                                                       (2048, 4096), (64, 16))
                                          if supported(m, rad, esz) and supported(n, rad, esz)])
def test_warp_group_cta_buffers_hold_their_pairs(mx, my, rad, esz):
    """Each group of G threads owns two buffers of `buf` complex values; the
    CTA's groups fit in the buffer region it is launched with."""
    lgx, lgy = (2 * mx).bit_length() - 1, (2 * my).bit_length() - 1
    gx, gy = geo32(lgx, rad), geo32(lgy, rad)
    threads = max(max(gx["G"], gy["G"]), 128)
    assert threads <= max_cta(rad, esz)
    region = max((threads // g["G"]) * 2 * g["buf"] for g in (gx, gy))
    for g in (gx, gy):
        groups = threads // g["G"]
        assert groups >= 1
        last = 2 * (groups - 1) * g["buf"] + 2 * g["buf"]
        assert last <= region


@pytest.mark.parametrize("mx,my,rad,esz", [(m, n, rad, esz) for rad in (8, 16, 32) for esz in (4, 8)
                                          for m, n in ((8, 8), (32, 64), (512, 1024), (1024, 512),
                                                       (2048, 4096), (64, 16), (16, 128))
                                          if supported(m, rad, esz) and supported(n, rad, esz)])
def test_joint_transposed_store_is_aligned_and_in_bounds(mx, my, rad, esz):
    """The x forward phase of a one-layer solve whose CTA holds two pairs
    (per == 2) writes both pairs' spectra as tr[k][r0 - 1 .. r0 + 2] when
    the two pairs cover four consecutive rows with (r0 - 1) % 4 == 0: every
    such piece lies inside the (mx + 1) x ld_tr plane and starts on 16
    bytes (ld_tr = round_up(my + 1, 32)); the other slots take the
    per-pair stores.  Every row 1 .. my - 1 is written by exactly one
    slot."""
    lgx, lgy = (2 * mx).bit_length() - 1, (2 * my).bit_length() - 1
    gx, gy = geo32(lgx, rad), geo32(lgy, rad)
    threads = max(max(gx["G"], gy["G"]), 128)
    per = threads // gx["G"]
    ld_tr = (my + 1 + 31) // 32 * 32
    nrows, ppl = my - 1, my // 2
    npairs = ppl
    nslots = (npairs + per - 1) // per
    rows = []

    def pair_rows(pair):
        pv = pair < npairs
        ra = 1 + 2 * (pair if pv else 0)
        return pv, ra, pv and ra + 1 <= nrows

    for slot in range(nslots):
        if per == 2:
            va0, r0, vb0 = pair_rows(2 * slot)
            va1, r1, vb1 = pair_rows(2 * slot + 1)
            if va0 and vb0 and va1 and vb1 and r1 == r0 + 2 and (r0 - 1) % 4 == 0:
                for k in range(1, gx["N"]):
                    off = k * ld_tr + (r0 - 1)
                    assert off + 3 < (mx + 1) * ld_tr
                    assert (off * esz) % 16 == 0
                rows += [r0, r0 + 1, r0 + 2, r0 + 3]
                continue
        for g in range(per):
            va, ra, vb = pair_rows(slot * per + g)
            if va:
                rows += [ra] + ([ra + 1] if vb else [])
    assert sorted(rows) == list(range(1, my))


def test_batched_solve_queue_claims_dependencies_first():
    """The batched solve's work items (phase by phase, member by member)
    decode to every (phase, member, slot) exactly once, and every item a
    phase-1 or phase-2 item waits for has a smaller index (so it was claimed
    earlier, by a running CTA)."""
    for nb, ns0, ns1 in itertools.product((1, 3, 7), (1, 2, 5), (1, 4)):
        n0, n1 = nb * ns0, nb * ns0 + nb * ns1
        total = n1 + nb * ns0
        seen = set()
        for item in range(total):
            if item < n0:
                ph, m, slot = 0, item // ns0, item % ns0
            elif item < n1:
                ph, m = 1, (item - n0) // ns1
                slot = item - n0 - m * ns1
            else:
                ph, m = 2, (item - n1) // ns0
                slot = item - n1 - m * ns0
            assert 0 <= m < nb and 0 <= slot < (ns1 if ph == 1 else ns0)
            seen.add((ph, m, slot))
            if ph > 0:
                prev = ([m * ns0 + s for s in range(ns0)] if ph == 1
                        else [n0 + m * ns1 + s for s in range(ns1)])
                assert max(prev) < item
        assert len(seen) == total


# ---- shared-memory Stockham engine (csrc/solve.cu, csrc/dst_engine.cuh) -------


def lane_cplx(N):
    return 2 * N + (N >> 3) + 2


def nb_for(N, E, max_threads=512):
    return max(1, (2 * N) // (E * max_threads))


def tpr_for(N, E):
    return (2 * N) // (E * nb_for(N, E))


def al16(v):
    return (v + 15) // 16 * 16


def stockham_layout_end(mx, my, esz, E):
    th = max(32, max(tpr_for(mx, E), tpr_for(my, E)))
    cx = 2 * esz
    bx, by = (th // tpr_for(mx, E)) * lane_cplx(mx), (th // tpr_for(my, E)) * lane_cplx(my)
    buf = al16(cx * max(bx, by))
    twx = 2 * mx * cx <= 32 * 1024
    twy = 2 * my * cx <= 32 * 1024
    lamy = buf
    tx = al16(lamy + esz * my)
    ty = al16(tx + (2 * mx * cx if twx else 0))
    return al16(ty + (2 * my * cx if twy else 0)), th


def stockham_supported(mx, my, esz, E):
    nbm = max(nb_for(mx, E), nb_for(my, E))
    return nbm <= 2 and stockham_layout_end(mx, my, esz, E)[0] <= 200 * 1024


# elliptic sides are at least 8 (qg_create rejects smaller grids; a level's
# grid is never smaller than the handle's), so L = 2N >= 16 >= E
SH = [(N, E) for E in (4, 16) for N in (8, 16, 32, 64, 256, 1024, 2048, 4096)
      if nb_for(N, E) <= 2]


@pytest.mark.parametrize("N,E", SH)
def test_stockham_engine_passes_and_extension(N, E):
    """The shared-memory engine's FFT of length L = 2N (base radix E, nb
    butterfly groups per thread, TPR threads per pair): each pass reads
    j + r L/R and writes (j - k) R + k + r Ns, both permutations of the L
    elements, inside the pair's padded lane of lane_cplx(N) slots; every
    twiddle index r k L/(R Ns) lies in the 2N-entry table; the odd
    extension writes every element of the sequence once."""
    L, nb = 2 * N, nb_for(N, E)
    TPR = L // (E * nb)
    assert TPR >= 1 and TPR * E * nb == L
    lg = L.bit_length() - 1
    if E == 16:
        passes = [(16, 16 ** p) for p in range(lg >> 2)]
        rem = lg & 3
        if rem:
            passes.append((1 << rem, 16 ** (lg >> 2)))
    else:
        passes = [(4, 4 ** p) for p in range(lg >> 1)]
        if lg & 1:
            passes.append((2, 4 ** (lg >> 1)))
    t = np.arange(TPR)
    for R, Ns in passes:
        per = E // R
        stride, tstep = L // R, L // (R * Ns)
        b = np.arange(nb * per)
        j = (t[:, None] + b[None, :] * TPR).ravel()
        k = j & (Ns - 1)
        r = np.arange(R)
        reads = j[:, None] + r[None, :] * stride
        writes = ((j - k) * R + k)[:, None] + r[None, :] * Ns
        for idx in (reads, writes):
            assert np.array_equal(np.sort(idx.ravel()), np.arange(L))
            assert px(idx.max()) < lane_cplx(N)
        if Ns > 1:
            assert (r.max() * k.max() * tstep) < 2 * N
    ext = [0, N] + [m for jj in range(1, N) for m in (jj, 2 * N - jj)]
    assert sorted(ext) == list(range(L))


@pytest.mark.parametrize("mx,my,esz,E", [(mx, my, esz, E) for E in (4, 16) for esz in (4, 8)
                                         for mx, my in ((8, 8), (32, 64), (64, 128), (256, 512),
                                                        (512, 1024), (1024, 2048), (2048, 4096),
                                                        (4096, 128))])
def test_stockham_engine_cta_fits(mx, my, esz, E):
    """Where the engine takes a grid, a CTA's threads hold whole pairs of
    both directions and its sequence lanes and tables fit the 200 KB it
    may use."""
    if not stockham_supported(mx, my, esz, E):
        return
    end, th = stockham_layout_end(mx, my, esz, E)
    assert end <= 200 * 1024 and th <= 512
    for N in (mx, my):
        assert th % tpr_for(N, E) == 0 and th // tpr_for(N, E) >= 1


# ---- long-sequence engine (csrc/solve_stream.cu, engine 50) -------------------


def sp(m):
    """Padded shared-memory slot of complex element m (one pad per 16)."""
    return m + (m >> 4)


def buf_elems(L):
    return sp(L) + 2


def stage_pitch(ppc):
    return 2 * ppc + (4 if ppc >= 4 else 2)


def tw_off(p):
    o, ns = 0, 16
    for _ in range(1, p):
        o += 16 * ns
        ns *= 16
    return o


def pass_table_size(L, rad):
    lg, lr = L.bit_length() - 1, rad.bit_length() - 1
    np_, rem = lg // lr, lg % lr
    n, ns = 0, rad
    for _ in range(1, np_):
        n += rad * ns
        ns *= rad
    if rem > 0 and np_ >= 1:
        n += (1 << rem) * ns
    return n


def ppc_for(lg, want, esz):
    p = want
    while p > 1 and (((1 << lg) // 16) * p > (1024 if esz == 4 else 512)
                     or p * buf_elems(1 << lg) * esz * 2 > 140 * 1024):
        p //= 2
    return p


STREAM = [(lg, esz) for esz in (4, 8) for lg in range(9, 15 if esz == 4 else 14)]


@pytest.mark.parametrize("lg,esz", STREAM)
def test_stream_engine_fft_slots_and_twiddles(lg, esz):
    """Engine 50's FFT of length L = 2^lg with G = L/16 threads of 16
    values: every pass's stores are a permutation of the L elements into
    padded slots below buf_elems(L), its loads read slot sp(element) (the
    per-thread base plus constant strides the kernel uses), the odd
    extension reads only slots written before it, and every twiddle read
    lies in the radix-16 pass table."""
    L, N, G = 1 << lg, 1 << (lg - 1), 1 << (lg - 4)
    NP, REM, LIM, SG = lg // 4, lg % 4, buf_elems(L), G + G // 16
    t, r = np.arange(G), np.arange(16)
    # loads t + r G at sp(t) + r sp(G)
    assert np.array_equal(sp(t)[:, None] + r[None, :] * SG, sp(t[:, None] + r[None, :] * G))
    # odd extension: stores z[t + r G] (r < 8) and the zero at N; loads
    # -z[c G - t], c = 16 - r, at c sp(G) - (t + ceil(t / 16))
    written = set(sp(t[:, None] + r[None, :8] * G).ravel().tolist()) | {sp(N)}
    assert max(written) < LIM
    u = t + ((t + 15) >> 4)
    for rr in range(8, 16):
        c = 16 - rr
        slot = c * SG - u
        assert np.array_equal(slot, sp(c * G - t))
        assert set(slot.tolist()) <= written
    # stores of the radix-16 passes (sub-transform size NS = 16^(p-1)) and
    # of the remainder pass (NS = 16^(NP-1))
    ns_list = [16 ** (p - 1) for p in range(1, NP)] + ([16 ** (NP - 1)] if REM else [])
    for NS in ns_list:
        if NS == 1:
            base, step = 17 * t, 1
            logical = 16 * t[:, None] + r[None, :]
        else:
            k = t & (NS - 1)
            d = (t - k) * 16 + k
            base, step = d + (d >> 4), NS + NS // 16
            logical = d[:, None] + r[None, :] * NS
        slots = base[:, None] + r[None, :] * step
        assert np.array_equal(slots, sp(logical))
        assert np.array_equal(np.sort(logical.ravel()), np.arange(L))
        assert slots.max() < LIM
    table = pass_table_size(L, 16)
    for P in range(1, NP):      # radix-16 pass P reads w, w^2, w^4, w^8 of its block
        NS = 16 ** P
        assert tw_off(P) + (NS - 1) + 8 * NS < table
    if REM:
        R = 1 << REM
        B, NSR = 16 // R, L // R
        b, rr = np.arange(B), np.arange(R)
        slots = (sp(t)[:, None, None] + b[None, :, None] * SG
                 + rr[None, None, :] * (NSR + NSR // 16))
        elems = t[:, None, None] + b[None, :, None] * G + rr[None, None, :] * NSR
        assert np.array_equal(slots, sp(elems))
        assert np.array_equal(np.sort(elems.ravel()), np.arange(L))
        assert tw_off(NP) + (G - 1) + (R - 1) * NSR < table


@pytest.mark.parametrize("lg,esz", STREAM)
@pytest.mark.parametrize("want", (1, 2, 4))
def test_stream_engine_staged_transposed_writes(lg, esz, want):
    """The passes that write transposed stage element k of group g's pair
    at [k SP + 2 g + (0, 1)] and write column q of rows k = k0 + i G/2 from
    thread e = k0 W + q: every (k, q) once, all inside the staging area,
    which with the FFT buffers fits the CTA's dynamic shared memory and the
    thread limit."""
    L, N, G = 1 << lg, 1 << (lg - 1), 1 << (lg - 4)
    ppc = ppc_for(lg, want, esz)
    threads = G * ppc
    assert threads <= (1024 if esz == 4 else 512)
    SP, W = stage_pitch(ppc), 2 * ppc
    grp = np.arange(ppc)
    k = np.arange(N)
    idx = k[:, None, None] * SP + 2 * grp[None, :, None] + np.arange(2)[None, None, :]
    assert idx.max() < N * SP
    assert len(set(idx.ravel().tolist())) == idx.size
    e = np.arange(threads)
    q, k0 = e % W, e // W
    KSTEP, ITER = G // 2, N // (G // 2)
    pairs = {(int(k0[j] + i * KSTEP), int(q[j])) for j in range(threads) for i in range(ITER)}
    assert pairs == {(kk, qq) for kk in range(N) for qq in range(W)}
    fft_bytes = ppc * buf_elems(L) * 2 * esz
    stg_bytes = N * SP * esz
    assert max(fft_bytes, stg_bytes) <= 227 * 1024
    assert fft_bytes <= 140 * 1024 or ppc == 1


# ---- mma.sync matrix-form solve (csrc/solve_mtx.cu, engine 40) ---------------


def mtx_geo(mx, my, layers=1):
    r16 = lambda v: (v + 15) // 16 * 16
    m, n = mx - 1, my - 1
    mp, np_ = r16(m), r16(n)
    ldx, ldy, lda, ldb = mp + 8, np_ + 4, mp + 4, mp + 8
    sx = 0
    sy = sx + mp * ldx
    u = sy + np_ * ldy
    v = u + np_ * ldb
    u2 = v + np_ * ldb
    v2 = u2 + np_ * ldb
    end = v2 + np_ * ldb if layers == 2 else u2
    return dict(m=m, n=n, mp=mp, np=np_, ldx=ldx, ldy=ldy, lda=lda, ldb=ldb, sx=sx, sy=sy, u=u,
                v=v, u2=u2, v2=v2, end=end, tinv=u, tend=u + np_ * mp)


def mtx_supported(mx, my, layers):
    return 2 <= mx <= 256 and 2 <= my <= 256 and mtx_geo(mx, my, layers)["end"] * 4 <= 200 * 1024


def mm3_reads(nrows, ncols, K, lda_, ldb_):
    """Largest A and B indices and the output cells of the 16 x 16-tile
    product: lane (q, t) of the warp of a tile reads A rows q, q + 8 at
    columns k0 + t, + 4 and B rows k0 + t, + 4 at columns q, q + 8 (+ 8 j);
    it writes rows q, q + 8 at columns 2t, 2t + 1 (+ 8 j)."""
    q, t = np.arange(8)[:, None], np.arange(4)[None, :]
    a_max = b_max = -1
    out = []
    for r0 in range(0, nrows, 16):
        for c0 in range(0, ncols, 16):
            for k0 in range(0, K, 8):
                a = (r0 + q + 8) * lda_ + k0 + t + 4
                b = (k0 + t + 4) * ldb_ + c0 + q + 8 * 1
                a_max, b_max = max(a_max, int(a.max())), max(b_max, int(b.max()))
            for j in range(2):
                c = c0 + 8 * j + 2 * t
                out.append(np.broadcast_to(r0 + q, (8, 4)) * 100000 + c)
                out.append(np.broadcast_to(r0 + q + 8, (8, 4)) * 100000 + c)
    return a_max, b_max, np.concatenate([o.ravel() for o in out])


MTX = [(mx, my, layers) for layers in (1, 2) for mx in (2, 4, 16, 32, 64, 128, 256)
       for my in (2, 8, 16, 32, 64, 128, 256) if mtx_supported(mx, my, layers)]


@pytest.mark.parametrize("mx,my,layers", MTX)
def test_matrix_engine_products_stay_in_their_operands(mx, my, layers):
    """The four products of the matrix-form solve (Q S_x, S_y (.) with the
    eigenvalue division, S_y (.), (.) S_x) read their A and B operands
    inside the operand's rows x pitch, write every (row, even column) pair
    of the np x mp output once with 8-byte-aligned float2 stores, and the
    operand regions are disjoint inside the CTA's shared memory; the
    table's S_x, S_y and Inv fit the table, and its bulk copies are 16-byte
    multiples at 16-byte offsets."""
    g = mtx_geo(mx, my, layers)
    mp, np_ = g["mp"], g["np"]
    assert g["end"] * 4 <= 200 * 1024
    regions = [(g["sx"], mp * g["ldx"]), (g["sy"], np_ * g["ldy"]), (g["u"], np_ * g["ldb"]),
               (g["v"], np_ * g["ldb"])]
    if layers == 2:
        regions += [(g["u2"], np_ * g["ldb"]), (g["v2"], np_ * g["ldb"])]
    for (a0, la), (b0, lb) in itertools.combinations(regions, 2):
        assert a0 + la <= b0 or b0 + lb <= a0
    assert max(a0 + la for a0, la in regions) <= g["end"]
    # (A, its pitch, its rows x columns, B, its pitch, its rows x columns, K)
    products = [
        (g["lda"], (np_, mp), g["ldx"], (mp, mp), mp),        # Q S_x -> V
        (g["ldy"], (np_, np_), g["ldb"], (np_, mp), np_),     # S_y V -> U (times Inv)
        (g["ldy"], (np_, np_), g["ldb"], (np_, mp), np_),     # S_y U -> V
        (g["lda"], (np_, mp), g["ldx"], (mp, mp), mp),        # V S_x -> psi
    ]
    for lda_, (ar, ac), ldb_, (br, bc), K in products:
        a_max, b_max, cells = mm3_reads(np_, mp, K, lda_, ldb_)
        assert ac <= lda_ and bc <= ldb_
        assert a_max < ar * lda_ and (a_max % lda_) < ac
        assert b_max < br * ldb_ and (b_max % ldb_) < bc
        assert len(np.unique(cells)) == cells.size == np_ * mp // 2
        for base, pitch in ((g["u"], g["ldb"]), (g["v"], g["ldb"]), (g["v"], g["lda"])):
            assert (base + pitch) % 2 == 0 and base % 2 == 0
    # Inv is read as float2 at r mp + c (c even) inside the table
    assert g["tinv"] + (np_ - 1) * mp + mp - 1 < g["tend"] and mp % 2 == 0
    for off, floats in ((g["sx"], mp * g["ldx"]), (g["sy"], np_ * g["ldy"])):
        assert (off * 4) % 16 == 0 and (floats * 4) % 16 == 0
    assert g["sy"] + np_ * g["ldy"] <= g["tinv"]


# ---- tcgen05 matrix-form solve (csrc/solve_tc.cu, engine 41) -----------------


def kmaj(r, k, K):
    """Byte offset of element (r, k) of a K-major operand without swizzle:
    8-row x 16-byte core matrices, 128 bytes apart along K, K/4 x 128 bytes
    apart along the rows."""
    return (r >> 3) * (K // 4) * 128 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4


def tc_geo(mx, my):
    r16 = lambda v: (v + 15) // 16 * 16
    m, n = mx - 1, my - 1
    mp, np_ = r16(m), r16(n)
    sx_half, sy_half = mp * mp * 4, 128 * np_ * 4
    op_half = max(128 * mp * 4, mp * np_ * 4)
    sx = 0
    sy = sx + 2 * sx_half
    op = sy + 2 * sy_half
    end = op + 2 * op_half
    c = max((mp // 8) * mp, (np_ // 8) * mp)
    cols = 32
    while cols < c:
        cols *= 2
    return dict(m=m, n=n, mp=mp, np=np_, sx=sx, sx_half=sx_half, sy=sy, sy_half=sy_half, op=op,
                op_half=op_half, end=end, cols=cols, tab_inv=op // 4)


TC = [(mx, my) for mx in (16, 32, 64) for my in (16, 32, 64)]


@pytest.mark.parametrize("mx,my", TC)
def test_tcgen05_operand_layout_and_budgets(mx, my):
    """The K-major layout is a bijection onto the operand's bytes; the
    descriptor of k-step ks (start ks x 256 bytes, leading offset 128 along
    K, stride offset K/4 x 128 along the rows) addresses element
    (r, 8 ks + kk) exactly where the layout put it; the operand regions are
    disjoint inside the CTA's shared memory; every product's K/8
    accumulators of N columns fit the TMEM allocation (a power of two, 32 ..
    512 columns); the instruction descriptor's fields hold M = 128 and N;
    the host table's split values and Inv lie inside it."""
    g = tc_geo(mx, my)
    mp, np_ = g["mp"], g["np"]
    for R, K in ((mp, mp), (128, np_), (128, mp), (mp, np_)):
        r, k = np.meshgrid(np.arange(R), np.arange(K), indexing="ij")
        off = kmaj(r, k, K)
        assert np.array_equal(np.sort(off.ravel()), 4 * np.arange(R * K))
        sbo = (K // 4) * 128
        for ks in range(K // 8):
            kk = np.arange(8)
            rr = np.arange(R)
            desc = (ks * 256 + (kk[None, :] // 4) * 128 + (rr[:, None] // 8) * sbo
                    + (rr[:, None] % 8) * 16 + (kk[None, :] % 4) * 4)
            assert np.array_equal(desc, kmaj(rr[:, None], 8 * ks + kk[None, :], K))
        assert sbo % 16 == 0 and (sbo >> 4) < (1 << 14)
    regions = [(g["sx"], 2 * g["sx_half"]), (g["sy"], 2 * g["sy_half"]), (g["op"], 2 * g["op_half"])]
    for (a0, la), (b0, lb) in itertools.combinations(regions, 2):
        assert a0 + la <= b0 or b0 + lb <= a0
    assert g["end"] <= 227 * 1024 and g["end"] % 16 == 0
    assert (g["sx_half"] >= mp * mp * 4 and g["sy_half"] >= 128 * np_ * 4
            and g["op_half"] >= max(128 * mp, mp * np_) * 4)
    assert g["cols"] in (32, 64, 128, 256, 512)
    for N, K in ((mp, mp), (mp, np_)):       # products 1 and 4; 2 and 3
        assert (K // 8 - 1) * N + N <= g["cols"]
        assert N % 8 == 0 and 8 <= N <= 256
        idesc = (1 << 4) | (2 << 7) | (2 << 10) | ((N >> 3) << 17) | ((128 >> 4) << 24)
        assert (idesc >> 17) & 0x3F == N >> 3 and (idesc >> 24) & 0x1F == 128 >> 4
    floats = g["tab_inv"] + np_ * mp
    top = max(max(g["sx"] + kmaj(i, kk, mp) + g["sx_half"] for i in range(g["m"]) for kk in (0, g["m"] - 1)),
              max(g["sy"] + kmaj(j, ll, np_) + g["sy_half"] for j in range(g["n"]) for ll in (0, g["n"] - 1)))
    assert top // 4 < g["tab_inv"]
    assert g["tab_inv"] + (g["n"] - 1) * mp + (g["m"] - 1) < floats


def queue_threads(lgx, esz):
    gy = (1 << (lgx + 1)) // 16
    maxt = 1024 if esz == 4 else 512
    return min(4 * gy, maxt)


@pytest.mark.parametrize("lgx,esz", [(lg, esz) for lg in (9, 10, 11) for esz in (4, 8)])
@pytest.mark.parametrize("nb", (1, 2, 12))
def test_stream_queue_items_and_shared_memory(lgx, esz, nb):
    """Engine 50's work queue for a batch of nb one-layer grids with
    my = 2 mx (2 mx = 2^lgx): items of PX x-pass pairs or PY y-pass pairs
    decode to every (pass, member, block) once, cover every pair of every
    member, and each item of pass 1 or 2 waits only for items numbered
    before it; one CTA size serves both lengths and its shared memory (FFT
    lanes or staging, whichever is larger) fits 227 KB."""
    L = 1 << lgx
    mx, my = L // 2, L
    BT = queue_threads(lgx, esz)
    Gx, Gy = L // 16, 2 * L // 16
    PX, PY = BT // Gx, BT // Gy
    assert PX >= 1 and PY >= 1 and PX * Gx == BT and PY * Gy == BT
    rows, cols = my // 2, mx // 2
    n0i, n1i = -(-rows // PX), -(-cols // PY)
    e0, e1 = nb * n0i, nb * n0i + nb * n1i
    total = e1 + nb * n0i
    seen, cover = set(), {0: set(), 1: set(), 2: set()}
    for item in range(total):
        if item < e0:
            ph, m = 0, item // n0i
            blk = item - m * n0i
        elif item < e1:
            ph, m = 1, (item - e0) // n1i
            blk = item - e0 - m * n1i
        else:
            ph, m = 2, (item - e1) // n0i
            blk = item - e1 - m * n0i
        assert 0 <= m < nb
        seen.add((ph, m, blk))
        per, npairs = (PY, cols) if ph == 1 else (PX, rows)
        for g in range(per):
            if blk * per + g < npairs:
                cover[ph].add((m, blk * per + g))
        if ph > 0:
            first_prev = e0 + m * n1i if ph == 2 else m * n0i
            nprev = n1i if ph == 2 else n0i
            assert first_prev + nprev - 1 < item
    assert len(seen) == total
    assert cover[0] == cover[2] == {(m, p) for m in range(nb) for p in range(rows)}
    assert cover[1] == {(m, p) for m in range(nb) for p in range(cols)}
    fft = max(PX * buf_elems(L), PY * buf_elems(2 * L)) * 2 * esz
    stg = max((L // 2) * stage_pitch(PX), L * stage_pitch(PY)) * esz
    assert max(fft, stg) <= 227 * 1024


# ---- multigrid (csrc/multigrid.cu, hierarchy in csrc/api.cu) -----------------


def padded_ld(n):
    return (n + 1 + 31) // 32 * 32


def mg_hierarchy(mx, my, esz, kmax_tail=14, tail_bytes=160 * 1024):
    """The grids (halved until the shorter side is 2 intervals), their
    pitches, and the first level of the one-CTA tail (the longest run of
    coarsest grids within the tail's shared-memory bound)."""
    xs, ys = [], []
    x, y = mx, my
    while True:
        xs.append(x)
        ys.append(y)
        if min(x, y) <= 2:
            break
        x, y = x // 2, y // 2
    nl = len(xs)

    def smem(k0):
        return sum(2 * (xs[k] + 1) * (ys[k] + 1) * esz for k in range(k0, nl))

    tail = nl - 1
    while tail > 0 and nl - tail < kmax_tail and smem(tail - 1) <= tail_bytes:
        tail -= 1
    return xs, ys, [padded_ld(v) for v in xs], tail, smem(tail)


def mg_supported(mx, my):
    lo, hi = min(mx, my), max(mx, my)
    return lo >= 2 and hi <= 4 * lo


MG = [(mx, my, esz) for esz in (4, 8) for mx, my in ((16, 32), (32, 64), (64, 128), (128, 256),
                                                     (256, 512), (512, 1024), (1024, 2048),
                                                     (2048, 4096), (64, 64), (128, 32), (8, 8))
      if mg_supported(mx, my)]


@pytest.mark.parametrize("mx,my,esz", MG)
def test_multigrid_indices(mx, my, esz):
    """Red-black half sweeps visit every interior point once per sweep and
    never two 4-neighbours in one colour (the in-place update has no race);
    restriction, prolongation and the 5-point stencils stay inside each
    grid's (my + 1) x ld array (pitch ld for the per-level grids, mx + 1 in
    the tail); the coarsest line has at most 8 unknowns (the line solve's
    array); the tail fits its shared memory."""
    xs, ys, lds, tail, tail_bytes = mg_hierarchy(mx, my, esz)
    assert tail_bytes <= 227 * 1024 and len(xs) - tail <= 14
    assert min(xs[-1], ys[-1]) == 2 and max(xs[-1], ys[-1]) - 1 <= 8
    for k, (gx, gy) in enumerate(zip(xs, ys)):
        for ld in ((lds[k], gx + 1) if k >= tail else (lds[k],)):
            assert ld >= gx + 1
            size = (gy + 1) * ld
            hw = gx // 2
            e = np.arange(hw * (gy - 1))
            jj = 1 + e // hw
            grids = []
            for color in (0, 1):
                ii = 2 * (e % hw) + np.where(((1 + jj) & 1) == color, 1, 2)
                keep = ii <= gx - 1
                i, j = ii[keep], jj[keep]
                if i.size:   # (a 2 x 2 grid has one point, of one colour)
                    assert i.min() >= 1 and j.min() >= 1 and j.max() <= gy - 1
                    o = j * ld + i
                    assert (o - ld).min() >= 0 and (o + ld).max() < size
                g = np.zeros((gy + 1, gx + 1), dtype=np.int32)
                np.add.at(g, (j, i), 1)
                assert g.max() <= 1                         # each point at most once
                b = g.astype(bool)
                # no two 4-neighbours of one colour
                assert not (b[:, 1:] & b[:, :-1]).any() and not (b[1:, :] & b[:-1, :]).any()
                grids.append(b)
            interior = np.zeros((gy + 1, gx + 1), dtype=bool)
            interior[1:gy, 1:gx] = True
            assert np.array_equal(grids[0] | grids[1], interior)
            assert not (grids[0] & grids[1]).any()
            if k + 1 < len(xs):
                cx_, cy_, cld = xs[k + 1], ys[k + 1], lds[k + 1] if k + 1 < tail else xs[k + 1] + 1
                assert cx_ == gx // 2 and cy_ == gy // 2
                # restriction: coarse (I, J) interior reads fine (2I +- 1, 2J +- 1)
                I = np.arange(1, cx_)
                J = np.arange(1, cy_)
                assert (2 * I + 1).max() <= gx - 1 and (2 * J + 1).max() <= gy - 1
                assert ((J.max()) * cld + I.max()) < (cy_ + 1) * cld
                # prolongation: fine (i, j) reads coarse (i >> 1 .. + 1, j >> 1 .. + 1)
                i = np.arange(1, gx)
                j = np.arange(1, gy)
                assert (i.max() >> 1) + 1 <= cx_ and (j.max() >> 1) + 1 <= cy_
                assert ((j.max() >> 1) + 1) * cld + (i.max() >> 1) + 1 < (cy_ + 1) * cld


# ---- diagnostics, adjoint, standalone transfers (diag.cu, adjoint.cu, stencil.cu)


DIAG = [(nx, ny) for nx, ny in ((8, 8), (64, 128), (512, 1024), (2048, 4096), (4096, 128))]


@pytest.mark.parametrize("nx,ny", DIAG)
def test_diagnostics_and_adjoint_indices(nx, ny):
    """The FP64 diagnostics walk nodes idx < nx ny (i = idx mod nx,
    j = idx / nx) and read psi at c + 1, c + ld (and c - 1, c - ld off the
    walls) inside the (ny + 1) x ld fine array; their edge sums take every
    x-edge of rows 1 .. ny - 1 and every y-edge of columns 1 .. nx - 1 once
    (the one-sided differences of the kinetic energy, walls zero).  The
    adjoint kernels' 32 x 8 blocks cover the interior, their 9-point
    stencils stay inside the array, and the dense accumulation is a
    bijection onto the (nx - 1)(ny - 1) exchange layout."""
    ld = padded_ld(nx)
    size = (ny + 1) * ld
    idx = np.arange(nx * ny)
    i, j = idx % nx, idx // nx
    c = j * ld + i
    assert (c + 1).max() < size and (c + ld).max() < size
    inner = (i >= 1) & (j >= 1)
    assert (c[inner] - ld).min() >= 0 and (c[inner] - 1).min() >= 0
    # the walk is a bijection onto the nodes (i, j) in [0, nx) x [0, ny), so
    # its j >= 1 part is every x-edge (i, j)-(i + 1, j) of rows 1 .. ny - 1
    # once, and its i >= 1 part every y-edge (i, j)-(i, j + 1) of columns
    # 1 .. nx - 1 once
    assert np.unique(c).size == nx * ny
    assert i.min() == 0 and i.max() == nx - 1 and j.min() == 0 and j.max() == ny - 1
    assert (j >= 1).sum() == nx * (ny - 1) and (i >= 1).sum() == (nx - 1) * ny
    bx, by = 32, 8
    gx, gy = (nx - 1 + bx - 1) // bx, (ny - 1 + by - 1) // by
    ii = np.arange(gx * bx) + 1
    jj = np.arange(gy * by) + 1
    assert ii.max() >= nx - 1 and jj.max() >= ny - 1
    I, J = np.meshgrid(ii[ii < nx], jj[jj < ny], indexing="ij")
    C = J * ld + I
    assert (C - ld - 1).min() >= 0 and (C + ld + 1).max() < size
    dense = (J - 1) * (nx - 1) + (I - 1)
    assert np.array_equal(np.sort(dense.ravel()), np.arange((nx - 1) * (ny - 1)))


@pytest.mark.parametrize("nx,ny,levels", [(nx, ny, lv) for nx, ny in ((64, 128), (512, 1024),
                                                                     (2048, 4096), (8192, 256))
                                          for lv in (1, 2, 3, 4) if (nx >> lv) >= 2 and (ny >> lv) >= 2])
def test_standalone_transfer_supports(nx, ny, levels):
    """Eq. res applied l times as one pass: coarse node (I, J), I in 1 ..
    mx - 1, reads fine nodes f I + di, f J + dj with |di|, |dj| < f = 2^l,
    all inside the fine grid's rows 0 .. ny and columns 0 .. nx (the walls
    contribute their zeros), and the hat weights (f - |d|) / f^2 sum to 1
    along each direction; Eq. pro applied l times reads coarse nodes
    (i >> l) .. + 1 inside the coarse array."""
    f = 1 << levels
    mx, my = nx >> levels, ny >> levels
    d = np.arange(-(f - 1), f)
    assert (f * 1 + d).min() >= 0 and (f * (mx - 1) + d).max() <= nx
    assert (f * 1 + d).min() >= 0 and (f * (my - 1) + d).max() <= ny
    assert np.sum(f - np.abs(d)) == f * f
    ldc = padded_ld(mx)
    i = np.arange(1, nx)
    j = np.arange(1, ny)
    assert (i.max() >> levels) + 1 <= mx and (j.max() >> levels) + 1 <= my
    assert ((j.max() >> levels) + 1) * ldc + (i.max() >> levels) + 1 < (my + 1) * ldc


# ---- fused fine-stage kernel (csrc/fused.cu) ---------------------------------

TX, SWX = 64, 72


def plan(esz, lv, tl, rc, ry=None):
    ry = ry if ry is not None else max(1 << lv, 8)
    G = rc // ry
    F = 1 << lv
    CPX, CPY = TX // F + 4, rc // F + 3

    def al(v):
        return (v + 127) // 128 * 128
    W = 0
    WN = al(W + esz * (rc + 2) * SWX)
    P = al(WN + esz * rc * TX)
    CP = al(P + (esz * (rc + 2) * SWX if lv == 0 else 0))
    CP2 = al(CP + (esz * CPY * CPX if lv > 0 else 0))
    FF = al(CP2 + (esz * CPY * CPX if tl else 0))
    END = al(FF + esz * rc * TX)
    return dict(RY=ry, G=G, THREADS=16 * G, F=F, CPX=CPX, CPY=CPY, END=END)


FUSED = ([(4, lv, False, rc, None) for lv in range(5) for rc in (128, 64, 32)]
         + [(4, lv, False, rc, 4) for lv in range(3) for rc in (64, 32)]
         + [(8, lv, False, 64, None) for lv in range(5)]
         + [(esz, lv, True, 128 if esz == 4 else 64, None) for esz in (4, 8) for lv in range(1, 5)])


@pytest.mark.parametrize("esz,lv,tl,rc,ry", FUSED)
def test_fused_tile_indices_stay_in_shared_memory(esz, lv, tl, rc, ry):
    pl = plan(esz, lv, tl, rc, ry)
    assert pl["RY"] % (1 << lv) == 0
    assert pl["END"] <= 200 * 1024                     # dynamic shared memory of a CTA
    assert rc % pl["RY"] == 0 and rc % pl["F"] == 0
    lanes = np.arange(16)
    # halo rows of w^(s) and of the fine psi: y - yc + 1 for the rows each
    # group touches, y in [ys - 1, ys + RY], ys = yc + grp RY
    for grp in range(pl["G"]):
        ys = grp * pl["RY"]
        rows = np.arange(ys - 1, ys + pl["RY"] + 1) + 1
        assert rows.min() >= 0 and rows.max() < rc + 2
    # the quad load (4 lane + 4 .. + 7) and the columns either side of it
    # (4 lane + 3, 4 lane + 8)
    assert (4 * lanes + 3).min() >= 0 and (4 * lanes + 8).max() < SWX
    # interior boxes (w^n, forcing): (y - yc) TX + 4 lane + 3 < RC TX
    assert (rc - 1) * TX + (4 * lanes + 3).max() < rc * TX
    if lv > 0:
        # the elliptic-grid patch: rows J - J_lo, columns Ib - I_lo .. + 3
        for x0, yc in ((0, 0), (TX, rc), (5 * TX, 7 * rc)):
            I_lo, J_lo = (x0 - 1) >> lv, (yc - 1) >> lv
            xq = x0 + 4 * lanes
            Ib = (xq - 1) >> lv
            cols = Ib - I_lo
            assert cols.min() >= 0 and (cols + 3).max() < pl["CPX"]
            for grp in range(pl["G"]):
                ys = yc + grp * pl["RY"]
                for y in range(ys - 1, ys + pl["RY"] + 1):
                    for J in (y >> lv, (y >> lv) + 1):
                        assert 0 <= J - J_lo < pl["CPY"]
        # the restriction's seam entries: 2 lane + 1 (l = 1), lane / G
        # (l >= 2) and TX / F, all < TX / F + 1
        sw = TX // pl["F"] + 1
        if lv == 1:
            assert (2 * lanes + 1).max() < sw
        else:
            gcell = max(pl["F"] // 4, 1)
            assert (lanes // gcell).max() < sw
        assert TX // pl["F"] < sw


@pytest.mark.parametrize("esz", [4, 8])
def test_fused_tma_boxes_start_on_16_bytes(esz):
    """The tile copies start at x = x0 - 4 (halo boxes) and x0 (interior
    boxes), x0 a multiple of 64 nodes: both multiples of 16 bytes."""
    for bx in range(0, 130):
        x0 = bx * TX
        assert ((x0 - 4) * esz) % 16 == 0 and (x0 * esz) % 16 == 0
