// Fused fine-grid stage of the one-layer model: prolongation on load,
// Arakawa / beta / dissipation / forcing and the TVDRK3 combination, and
// restriction on store, in one pass over the fine grid.
//
// A CTA covers a 64-node-wide column block over RC = GROUPS x 16 rows.  One
// elected thread stages its inputs into shared memory with 2-D TMA tensor
// copies (w^(s) with a halo, w^n, the fine psi for l = 0, a forcing field),
// all issued at once and completed on one mbarrier, so a CTA keeps its whole
// working set (~70 KB) in flight; the wait is bounded and a timeout sets an
// error flag instead of hanging.  Meanwhile the other threads stage the
// elliptic-grid streamfunction patch.  Then each group of 16 threads (half a
// warp) owns the block's columns,
// x in [x0, x0 + 64), 4 x-consecutive nodes per thread, and sweeps the 16
// fine rows y in [ys, ys + 16), ys a multiple of 16, keeping the three rows
// of w^(s) and psi its stencil needs in registers.  x-halos come from the
// neighbouring threads by shuffles (the group's first and last thread read
// the block's edge columns).  Per row it
//   1. loads w^(s) of the next row, and builds psi of that row either by
//      bilinear interpolation from the elliptic-grid streamfunction held in
//      registers (Eq. pro applied l times is bilinear interpolation at
//      2^-l spacing) or, for l = 0, by loading the fine psi;
//   2. computes w^(s+1) = a w^n + b (w^(s) + dt G) with
//      G = -J(psi, w) - (1/Ro) J(psi, y) + (1/Re) lap w + F (Eqs. ja1, j1-j3,
//      Eq. ge divided by Ro) and stores it;
//   3. for l >= 1 adds the row's share to the restriction of w^(s+1):
//      Eq. res applied l times has the separable hat weights (f-|d|)/f^2,
//      f = 2^l, so a node at distance d in [0, f) past coarse line N gives
//      (f-d)/f^2 of itself to N and d/f^2 to N+1 in each direction; the x
//      shares are combined across threads by shuffles and the y shares
//      accumulate in registers over the sweep.
// A coarse node whose support straddles the block's right edge line or the
// group's last row receives the rest from the neighbouring block or group,
// so each group writes its sums into one of four planes by the node's
// position (q = 0: the node lies in the group's block and rows; bit 0: on
// the block's right edge line; bit 1: on the row after the group's last).
// Every (node, plane) has one writer, planes 1-3 stay zero off those lines,
// and the row sine transform adds P0 + P1 + P2 + P3 in that order.
#include <cuda_runtime.h>

#include <type_traits>

#include "bounds.cuh"
#include "qg_internal.cuh"

namespace qg {
namespace {

constexpr int TX = 64;      // nodes per column block (16 threads x 4)
constexpr int SWX = TX + 8; // halo tile row: fine x in [x0 - 4, x0 + 68)
// rows swept by one group: 8, or 2^l when that is larger (a group must
// cover whole coarse cells for the partial-sum planes)
template <int LV> struct Sweep { static constexpr int RY = (1 << LV) > 8 ? (1 << LV) : 8; };

// fine rows per CTA: FP32 one-layer sweeps are built for 128, 64 and 32
// (the autotuner picks one per handle); FP64 and two-layer sweeps use 64
// and 128 rows
template <typename T> struct Rows { static constexpr int value = 128; };
template <> struct Rows<double> { static constexpr int value = 64; };

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T v[4]) {
    v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
}
__device__ __forceinline__ void lds4(const float* p, float v[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void lds4(const double* p, double v[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void stg4(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void stg4(double* p, const double v[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *(reinterpret_cast<double2*>(p) + 1) = make_double2(v[2], v[3]);
}

// ---- mbarrier / TMA (inline PTX) --------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Bounded wait for phase `parity` of the barrier: true when it completed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Shared-memory plan of one CTA (byte offsets, 128-byte aligned).
template <typename T, int LV, bool TL = false, int RC_ = Rows<T>::value, int RY_ = Sweep<LV>::RY>
struct Plan {
    static constexpr int RC = RC_;
    static constexpr int RY = RY_;                  // fine rows swept by one thread
    static_assert(RY % (1 << LV) == 0 && RC % RY == 0, "a group covers whole coarse cells");
    static constexpr int G = RC / RY;               // groups per CTA
    static constexpr int THREADS = 16 * G;
    // CTAs per SM the registers are budgeted for: FP32 one-layer sweeps as
    // many as make 640 threads (102 registers each: at 80, for 768 threads,
    // the l >= 1 sweeps spill); FP64 and two-layer sweeps 2 CTAs (their
    // state needs up to 232 registers)
    static constexpr int MINB_RAW = (sizeof(T) == 4 && !TL) ? 640 / THREADS : 2;
    static constexpr int MINB = MINB_RAW < 1 ? 1 : (MINB_RAW > 16 ? 16 : MINB_RAW);
    static constexpr int F = 1 << LV;
    static constexpr int CPX = TX / F + 4;
    static constexpr int CPY = RC / F + 3;
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t W = 0;                                             // (RC+2) x SWX
    static constexpr size_t WN = al(W + sizeof(T) * (RC + 2) * SWX);          // RC x TX
    static constexpr size_t P = al(WN + sizeof(T) * RC * TX);                 // (RC+2) x SWX (l = 0)
    static constexpr size_t CP = al(P + (LV == 0 ? sizeof(T) * (RC + 2) * SWX : 0));  // l >= 1
    static constexpr size_t CP2 = al(CP + (LV > 0 ? sizeof(T) * CPY * CPX : 0));      // two layers
    static constexpr size_t FF = al(CP2 + (TL ? sizeof(T) * CPY * CPX : 0));          // RC x TX
    static constexpr size_t END_NOF = FF;                 // without a forcing field
    static constexpr size_t END = al(FF + sizeof(T) * RC * TX);
};

// The work of one CTA: the tile (bx, by) of one basin, whose tensor maps and
// parameters the two kernels below take from the launch (one basin) or from
// a table in device memory (a batch of ensemble members).
template <typename T, int LV, bool TL, int RCT, int RYT = Sweep<LV>::RY>
__device__ __forceinline__ void sweep_tile(const CUtensorMap* tm_w, const CUtensorMap* tm_wn,
                                           const CUtensorMap* tm_p, const CUtensorMap* tm_f,
                                           const FusedParams<T>& p, int bx, int by) {
    using PL = Plan<T, LV, TL, RCT, RYT>;
    constexpr int F = 1 << LV;
    constexpr int RC = PL::RC;
    constexpr int RY = PL::RY;
    constexpr int NM = RY / F + 1;                  // node rows a group touches
    constexpr int G = (F >= 4) ? F / 4 : 1;          // threads per coarse cell
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    // restriction partial sums of node rows on the seam between two groups
    __shared__ T seam[(LV > 0) ? PL::G : 1][(LV > 0) ? TX / (1 << LV) + 1 : 1];
    T* sw = reinterpret_cast<T*>(smem + PL::W);
    T* swn = reinterpret_cast<T*>(smem + PL::WN);
    T* sp = reinterpret_cast<T*>(smem + PL::P);
    T* sf = reinterpret_cast<T*>(smem + PL::FF);
    T* cp = reinterpret_cast<T*>(smem + PL::CP);
    T* cp2 = reinterpret_cast<T*>(smem + PL::CP2);   // the other layer's psi (two layers)

    const int nx = p.nx, ny = p.ny, ld = p.ld;
    const int x0 = bx * TX;
    const int yc = by * RC;
    const bool use_wn = p.a != T(0);
    const bool use_f = p.f2d != nullptr;
    const uint32_t bar = smem_u32(&mbar);

    // ---- stage the inputs ------------------------------------------------
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // w^(s), w^n and the forcing were written before the solve this kernel
    // follows began (the solve is launched in stream order), so their copies
    // start before the programmatic wait; psi comes from the solve itself.
    if (threadIdx.x == 0) {
        uint32_t bytes = sizeof(T) * (RC + 2) * SWX;
        if (use_wn) bytes += sizeof(T) * RC * TX;
        if (LV == 0) bytes += sizeof(T) * (RC + 2) * SWX;
        if (use_f) bytes += sizeof(T) * RC * TX;
        mbar_expect_tx(bar, bytes);
        // box x coordinates are multiples of 16 bytes (x0 is a multiple of
        // 64 nodes, the halo box starts 4 nodes left of it)
        if (QG_IN(((x0 - 4) * (int)sizeof(T)) & 15, 1, 1))
            tma_load_2d(smem_u32(sw), tm_w, x0 - 4, yc - 1, bar);
        if (use_wn && QG_IN((x0 * (int)sizeof(T)) & 15, 1, 2))
            tma_load_2d(smem_u32(swn), tm_wn, x0, yc, bar);
        if (use_f && QG_IN((x0 * (int)sizeof(T)) & 15, 1, 3))
            tma_load_2d(smem_u32(sf), tm_f, x0, yc, bar);
    }
    pdl_wait();
    if (LV == 0 && threadIdx.x == 0) tma_load_2d(smem_u32(sp), tm_p, x0 - 4, yc - 1, bar);
    // the step size: fixed, or Eq. dt from this step's first streamfunction
    // (one FP64 division per CTA, shared through the barrier below)
    __shared__ T s_dt;
    if (threadIdx.x == 0) {
        double dtd = (double)p.dt;
        if (p.umax) {
            const double u = __longlong_as_double((long long)*p.umax);
            dtd = u > 0.0 ? fmin(p.dt_cap, p.cfl_h / u) : p.dt_cap;
        }
        s_dt = (T)dtd;
        if (p.last_stage && bx == 0 && by == 0) {
            p.clock[0] += dtd;
            p.clock[1] = dtd;
        }
    }
    const int mx = nx >> LV, my = ny >> LV;
    const int I_lo = (x0 - 1) >> LV;      // may be -1
    const int J_lo = (yc - 1) >> LV;      // may be -1
    if (LV > 0) {
        for (int e = threadIdx.x; e < PL::CPX * PL::CPY; e += blockDim.x) {
            const int ii = e % PL::CPX, jj = e / PL::CPX;
            const int I = I_lo + ii, J = J_lo + jj;
            const bool in = I >= 0 && I <= mx && J >= 0 && J <= my &&
                            QG_IN((long long)J * p.ldp + I, (long long)(my + 1) * p.ldp, 4);
            cp[e] = in ? __ldg(p.psi + (size_t)J * p.ldp + I) : T(0);
            if constexpr (TL) cp2[e] = in ? __ldg(p.psi_o + (size_t)J * p.ldp + I) : T(0);
        }
    }
    const bool arrived = mbar_wait(bar, 0, kWaitLimit);
    __syncthreads();
    if (!arrived) {
        if (threadIdx.x == 0) atomicExch(p.err, 1);
        (void)mbar_wait(bar, 0, kWaitLimit);     // let copies in flight land
        return;
    }
    const T dt = s_dt;

    // ---- sweep -----------------------------------------------------------
    const int lane = threadIdx.x & 15;
    const int grp = threadIdx.x >> 4;
    const unsigned gm = 0xFFFFu << (16 * (grp & 1));
    const int ys = yc + grp * RY;
    const bool active = ys < ny;                     // uniform in the group
    const int xq = x0 + 4 * lane;

    // row y of a halo tile (w^(s) or the fine psi): own quad and the
    // columns either side, all in the tile
    auto row_halo = [&](const T* tile, int y, T v[6]) {
        const int o = (y - yc + 1) * SWX + 4 * lane;
        const T* r = tile + o;
        T c[4] = {T(0), T(0), T(0), T(0)};
        const bool ok = QG_IN(o + 8, (RC + 2) * SWX, 5) && QG_IN(o + 3, (RC + 2) * SWX, 5);
        if (ok) lds4(r + 4, c);
        v[0] = ok ? r[3] : T(0);
        v[1] = c[0]; v[2] = c[1]; v[3] = c[2]; v[4] = c[3];
        v[5] = ok ? r[8] : T(0);
    };
    const int Ib = (xq - 1) >> LV;
    T c0[4], c1[4], d0[4], d1[4];    // coarse rows around y of psi (and of the other layer)
    auto coarse_row = [&](const T* patch, int J, T (&c)[4]) {
        const T* r = patch + (J - J_lo) * PL::CPX + (Ib - I_lo);
        const int o = (J - J_lo) * PL::CPX + (Ib - I_lo);
        const bool ok = QG_IN(o, PL::CPX * PL::CPY, 6) && QG_IN(o + 3, PL::CPX * PL::CPY, 6);
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = ok ? r[k] : T(0);
    };
    // ph = y mod 2^l, known at compile time in the unrolled sweep (ys is a
    // multiple of RY, itself a multiple of 2^l).  Sums of products are
    // written as explicit fma: left to the compiler, the two instantiations
    // of this body (one basin, batch) could contract them differently.
    auto psi_row = [&](int y, int ph, const T (&c0)[4], const T (&c1)[4], T v[6], bool chk) {
        if (chk && (y < 0 || y >= ny)) {
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = T(0);
            return;
        }
        const T b = T(ph) * (T(1) / T(F));
        T cv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cv[k] = ph == 0 ? c0[k] : fma(b, c1[k], (T(1) - b) * c0[k]);
        if (LV == 1) {
            v[0] = T(0.5) * (cv[0] + cv[1]); v[1] = cv[1];
            v[2] = T(0.5) * (cv[1] + cv[2]); v[3] = cv[2];
            v[4] = T(0.5) * (cv[2] + cv[3]); v[5] = cv[3];
        } else if (LV == 2) {
            v[0] = fma(T(0.75), cv[1], T(0.25) * cv[0]); v[1] = cv[1];
            v[2] = fma(T(0.25), cv[2], T(0.75) * cv[1]);
            v[3] = T(0.5) * (cv[1] + cv[2]);
            v[4] = fma(T(0.75), cv[2], T(0.25) * cv[1]); v[5] = cv[2];
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int x = xq - 1 + k;
                const int cell = (x >> LV) - Ib;
                const T a = T(x & (F - 1)) * (T(1) / T(F));
                const T lo = cell == 0 ? cv[0] : (cell == 1 ? cv[1] : cv[2]);
                const T hi = cell == 0 ? cv[1] : (cell == 1 ? cv[2] : cv[3]);
                v[k] = fma(a, hi, (T(1) - a) * lo);
            }
        }
        // columns at or beyond a wall interpolate between the zero wall
        // values and the zero fill of the patch, so they come out zero
    };
    // psi of sweep row rr (fine row y = ys - 1 + rr), and for two layers
    // the other layer's psi of that row
    auto load_psi = [&](int rr, int y, T v[6], T* vo, bool chk) {
        if (LV == 0) {
            row_halo(sp, y, v);
        } else {
            if (rr <= 1) {
                coarse_row(cp, y >> LV, c0);
                coarse_row(cp, (y >> LV) + 1, c1);
                if constexpr (TL) {
                    coarse_row(cp2, y >> LV, d0);
                    coarse_row(cp2, (y >> LV) + 1, d1);
                }
            } else if (((rr - 1) & (F - 1)) == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) c0[k] = c1[k];
                coarse_row(cp, (y >> LV) + 1, c1);
                if constexpr (TL) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) d0[k] = d1[k];
                    coarse_row(cp2, (y >> LV) + 1, d1);
                }
            }
            const int ph = (rr - 1) & (F - 1);
            psi_row(y, ph, c0, c1, v, chk);
            if constexpr (TL) psi_row(y, ph, d0, d1, vo, chk);
        }
    };
    // two layers: w_i = Q_i/Ro + k_p (psi_i - psi_j) on a row (Eq. pv-non)
    auto w_row = [&](const T q[6], const T ps[6], const T po[6], T v[6]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = fma(p.k_p, ps[k] - po[k], p.inv_Ro * q[k]);
    };

    T accA[NM], accB[NM], accE[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) accA[m] = accB[m] = accE[m] = T(0);
    // A tile that touches no wall (its rows, the rows above and below it
    // and its columns all interior) sweeps without the per-row wall tests:
    // one-layer FP32 sweeps at l <= 2, where the second body costs no
    // spills.  (A third body for stages without w^n measured slower.)
    constexpr bool kSplit = sizeof(T) == 4 && !TL && LV <= 2;
    const bool interior = kSplit && x0 >= 1 && x0 + TX <= nx && yc >= 1 && yc + RC <= ny - 1;
    auto sweep = [&](auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;
        // rows y-1, y, y+1 of w^(s) and psi in rotating slots (two layers:
        // also the relative vorticity WV of the dissipation)
        T W[3][6], P[3][6], WV[TL ? 3 : 1][6], PO[TL ? 6 : 1];
        row_halo(sw, ys - 1, W[0]);
        load_psi(0, ys - 1, P[0], PO, !IN);
        if constexpr (TL) w_row(W[0], P[0], PO, WV[0]);
        row_halo(sw, ys, W[1]);
        load_psi(1, ys, P[1], PO, !IN);
        if constexpr (TL) w_row(W[1], P[1], PO, WV[1]);
        // w^(s+1) = a w^n + b w^(s) + b dt G: the coefficients of G come
        // scaled by b dt, and for one layer the centre weight of the
        // Laplacian joins b on w^(s)
        const T c_lap0 = T(-2) * (p.c_lapx + p.c_lapy);
        const T bdt = p.b * dt;
        const T k_beta = -p.c_beta * bdt, k_jac = -p.c_jac * bdt;
        const T k_lx = p.c_lapx * bdt, k_ly = p.c_lapy * bdt;
        const T k_0 = TL ? (c_lap0 - p.drag) * bdt : fma(c_lap0, bdt, p.b);

    #pragma unroll
        for (int o = 0; o < RY; ++o) {
            const int y = ys + o;
            const int sb = o % 3, sc = (o + 1) % 3, sa = (o + 2) % 3;
            row_halo(sw, y + 1, W[sa]);
            load_psi(o + 2, y + 1, P[sa], PO, !IN);
            if constexpr (TL) w_row(W[sa], P[sa], PO, WV[sa]);
            const bool row_ok = IN || (y >= 1 && y <= ny - 1);
            const size_t ro = (size_t)y * ld;
            T wn[4] = {T(0), T(0), T(0), T(0)};
            const bool row_in = QG_IN((y - yc) * TX + 4 * lane + 3, RC * TX, 7) &&
                                QG_IN((y - yc) * TX, RC * TX, 7);
            if (use_wn && row_in) lds4(swn + (y - yc) * TX + 4 * lane, wn);
            T fv[4] = {T(0), T(0), T(0), T(0)};
            if (use_f) {
                if (row_in) lds4(sf + (y - yc) * TX + 4 * lane, fv);
            } else {
                // (the bottom layer of two has no wind: frow is null there)
                const T fr = (!TL || p.frow) ? __ldg(p.frow + (IN || y <= ny ? y : ny)) : T(0);
    #pragma unroll
                for (int q = 0; q < 4; ++q) fv[q] = fr;
            }
            // differences shared by the four nodes: vertical psi differences
            // V_c per column and their neighbour sums S_c = V_c + V_{c+1};
            // horizontal differences H of rows y-1, y, y+1 and the sums
            // Ta = H(y+1) + H(y), Tb = H(y) + H(y-1)
            T V[6], S[5], Ha[4], Hb[4], Hc[4], Ta[4], Tb[4];
    #pragma unroll
            for (int c = 0; c < 6; ++c) V[c] = P[sa][c] - P[sb][c];
    #pragma unroll
            for (int c = 0; c < 5; ++c) S[c] = V[c] + V[c + 1];
    #pragma unroll
            for (int q = 0; q < 4; ++q) {
                Ha[q] = P[sa][q + 2] - P[sa][q];
                Hb[q] = P[sb][q + 2] - P[sb][q];
                Hc[q] = P[sc][q + 2] - P[sc][q];
                Ta[q] = Ha[q] + Hc[q];
                Tb[q] = Hc[q] + Hb[q];
            }
            T out[4];
    #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = q + 1;
                const T pm0 = P[sc][i - 1], p10 = P[sc][i + 1], p0m = P[sb][i], p01 = P[sa][i];
                const T q00 = W[sc][i];
                const T qm0 = W[sc][i - 1], q10 = W[sc][i + 1], q0m = W[sb][i], q01 = W[sa][i];
                const T qmm = W[sb][i - 1], q1m = W[sb][i + 1], qm1 = W[sa][i - 1], q11 = W[sa][i + 1];
                // Arakawa J1 + J2 + J3 (Eqs. j1-j3) gathered by neighbour of q:
                //   edge neighbours (J1 + J2): -q10 (V_i + V_{i+1}) + qm0 (V_{i-1} + V_i)
                //                              + q01 (Hc + Ha) - q0m (Hc + Hb)
                //   corners (J3): -q11 (p01 - p10) + qmm (pm0 - p0m)
                //                 + qm1 (p01 - pm0) - q1m (p10 - p0m)
                T jac = -q10 * S[i];
                jac = fma(qm0, S[i - 1], jac);
                jac = fma(q01, Ta[q], jac);
                jac = fma(-q0m, Tb[q], jac);
                jac = fma(-q11, p01 - p10, jac);
                jac = fma(qmm, pm0 - p0m, jac);
                jac = fma(qm1, p01 - pm0, jac);
                jac = fma(-q1m, p10 - p0m, jac);
                // (1/Ro) J(psi, y) in Arakawa's form: (4 c_j + c_{j+1} + c_{j-1})/(6 Ro)
                const T beta = fma(T(4), Hc[q], Ha[q] + Hb[q]);
                // b dt G, G = F + (1/Re) lap w - J(psi, w)/(12 dx dy) - beta/(12 Ro dx)
                T Gv = fma(k_beta, beta, bdt * fv[q]);
                Gv = fma(k_jac, jac, Gv);
                if constexpr (TL) {
                    // A lap w_i - drag w_i (Eq. ge-non)
                    const T v00 = WV[sc][i];
                    Gv = fma(k_0, v00, Gv);
                    Gv = fma(k_ly, WV[sa][i] + WV[sb][i], Gv);
                    Gv = fma(k_lx, WV[sc][i + 1] + WV[sc][i - 1], Gv);
                    Gv = fma(p.b, q00, Gv);
                } else {
                    Gv = fma(k_0, q00, Gv);
                    Gv = fma(k_ly, q01 + q0m, Gv);
                    Gv = fma(k_lx, q10 + qm0, Gv);
                }
                out[q] = fma(p.a, wn[q], Gv);
            }

            const bool quad_ok = IN || (row_ok && xq >= 1 && xq + 3 <= nx - 1);
            const long long fine_n = (long long)(ny + 1) * ld;
            if (quad_ok) {
                if (QG_IN(ro + xq + 3, fine_n, 8)) stg4(p.wout + ro + xq, out);
            } else {
    #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int x = xq + q;
                    if (row_ok && x >= 1 && x <= nx - 1) {
                        if (QG_IN(ro + x, fine_n, 8)) p.wout[ro + x] = out[q];
                    } else {
                        out[q] = T(0);
                    }
                }
            }
            if (LV > 0) {
                // x shares of this row
                T xa, xb = T(0), xe;
                if (LV == 1) {
                    const T A = fma(T(0.25), out[1], T(0.5) * out[0]);
                    const T C = T(0.25) * out[3];
                    xb = fma(T(0.25), out[3], fma(T(0.5), out[2], T(0.25) * out[1]));
                    const T Cp = __shfl_up_sync(gm, C, 1, 16);
                    xa = A + (lane > 0 ? Cp : T(0));
                    xe = C;
                } else {
                    T Va = T(0), Vb = T(0);
    #pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // x0 is a multiple of 64 and xq of 4
                        const int d = F <= 4 ? (q & (F - 1)) : ((4 * lane + q) & (F - 1));
                        Va += T(F - d) * (T(1) / T(F * F)) * out[q];
                        Vb += T(d) * (T(1) / T(F * F)) * out[q];
                    }
    #pragma unroll
                    for (int off = 1; off < G; off <<= 1) {
                        Va += __shfl_xor_sync(gm, Va, off, 16);
                        Vb += __shfl_xor_sync(gm, Vb, off, 16);
                    }
                    const T Vbp = __shfl_up_sync(gm, Vb, G, 16);
                    xa = Va + (lane >= G ? Vbp : T(0));
                    xe = Vb;
                }
                const int dy = o & (F - 1);
                const int mlo = o >> LV;
                const T wlo = T(F - dy) * (T(1) / T(F * F));
                const T whi = T(dy) * (T(1) / T(F * F));
                accA[mlo] += wlo * xa;
                accE[mlo] += wlo * xe;
                if (LV == 1) accB[mlo] += wlo * xb;
                if (dy != 0) {
                    accA[mlo + 1] += whi * xa;
                    accE[mlo + 1] += whi * xe;
                    if (LV == 1) accB[mlo + 1] += whi * xb;
                }
            }
        }
    };
    if (active) {
        if constexpr (kSplit) {
            if (interior)
                sweep(std::true_type{});
            else
                sweep(std::false_type{});
        } else {
            sweep(std::false_type{});
        }
    }
    pdl_trigger();
    // ---- restriction partial sums ---------------------------------------
    // The node row on the seam between group g and g+1 of this CTA gets its
    // two shares added here (lower group's share first); only the last
    // group's top row, on the CTA's seam, goes to a seam plane.
    if (LV > 0) {
        constexpr int SW = TX / (1 << LV) + 1;   // seam entries per group
        if (active) {
            if (LV == 1) {
                if (QG_IN(2 * lane + 1, SW, 9)) {
                    seam[grp][2 * lane] = accA[NM - 1];
                    seam[grp][2 * lane + 1] = accB[NM - 1];
                }
            } else if (lane % G == 0) {
                if (QG_IN(lane / G, SW, 9)) seam[grp][lane / G] = accA[NM - 1];
            }
            if (lane == 15) seam[grp][TX / F] = accE[NM - 1];
        }
        __syncthreads();
        if (active && grp > 0) {
            if (LV == 1) {
                accA[0] = seam[grp - 1][2 * lane] + accA[0];
                accB[0] = seam[grp - 1][2 * lane + 1] + accB[0];
            } else if (lane % G == 0) {
                accA[0] = seam[grp - 1][lane / G] + accA[0];
            }
            if (lane == 15) accE[0] = seam[grp - 1][TX / F] + accE[0];
        }
        if (active) {
            const int Ix0 = x0 >> LV;
            const int mlast = (grp == PL::G - 1) ? NM : NM - 1;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                if (m >= mlast) break;
                const int J = (ys >> LV) + m;
                if (J < 1 || J > my - 1) continue;
                const int qy = (m == NM - 1) ? 2 : 0;
                T* rowA = p.part[qy] + (size_t)J * p.ldc;
                const long long pn = (long long)(my + 1) * p.ldc;
                const long long jo = (long long)J * p.ldc;
                if (LV == 1) {
                    const int I = Ix0 + 2 * lane;
                    if (I >= 1 && I <= mx - 1 && QG_IN(jo + I, pn, 10)) rowA[I] = accA[m];
                    if (I + 1 >= 1 && I + 1 <= mx - 1 && QG_IN(jo + I + 1, pn, 10))
                        rowA[I + 1] = accB[m];
                } else if (lane % G == 0) {
                    const int I = Ix0 + lane / G;
                    if (I >= 1 && I <= mx - 1 && QG_IN(jo + I, pn, 10)) rowA[I] = accA[m];
                }
                if (lane == 15) {
                    const int I = Ix0 + TX / F;
                    if (I >= 1 && I <= mx - 1 && QG_IN(jo + I, pn, 10))
                        p.part[qy + 1][(size_t)J * p.ldc + I] = accE[m];
                }
            }
        }
    }
}

template <typename T, int LV, bool TL, int RCT, int RYT>
__global__ void __launch_bounds__(Plan<T, LV, TL, RCT, RYT>::THREADS,
                                  Plan<T, LV, TL, RCT, RYT>::MINB)
fine_sweep_kernel(const __grid_constant__ CUtensorMap tm_w,
                  const __grid_constant__ CUtensorMap tm_wn,
                  const __grid_constant__ CUtensorMap tm_p,
                  const __grid_constant__ CUtensorMap tm_f, FusedParams<T> p) {
    sweep_tile<T, LV, TL, RCT, RYT>(&tm_w, &tm_wn, &tm_p, &tm_f, p, blockIdx.x, blockIdx.y);
}

// Batched fine stage of an ensemble: CTA c sweeps tile (tiles[c].y,
// tiles[c].z) of member tiles[c].x; the member's tensor maps and parameters
// are read from `fm` in device memory (written by the host before the
// launch).  One layer only.
template <typename T, int LV, int RCT>
__global__ void __launch_bounds__(Plan<T, LV, false, RCT>::THREADS, Plan<T, LV, false, RCT>::MINB)
fine_batch_kernel(const FineMember<T>* __restrict__ fm, const int4* __restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const FineMember<T>* E = fm + t.x;
    if (threadIdx.x == 0) {
        // the tensor maps live in global memory: order the copy proxy's reads
        // of them after the host's writes
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&E->w) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&E->wn) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&E->psi) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&E->f) : "memory");
    }
    sweep_tile<T, LV, false, RCT>(&E->w, &E->wn, &E->psi, &E->f, E->p, t.y, t.z);
}

template <typename T, int LV, int RCT>
cudaError_t launch_batch(const FineMember<T>* fm, const int4* tiles, int ntiles, bool forcing_field,
                         bool pdl, cudaStream_t s) {
    using PL = Plan<T, LV, false, RCT>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fine_batch_kernel<T, LV, RCT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)PL::END);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntiles);
    cfg.blockDim = dim3(PL::THREADS);
    cfg.dynamicSmemBytes = forcing_field ? PL::END : PL::END_NOF;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fine_batch_kernel<T, LV, RCT>, fm, tiles);
}

template <typename T, int LV, bool TL, int RCT, int RYT = Sweep<LV>::RY>
cudaError_t launch_sweep(const FusedParams<T>& p, const FineMaps& m, cudaStream_t s) {
    using PL = Plan<T, LV, TL, RCT, RYT>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fine_sweep_kernel<T, LV, TL, RCT, RYT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)PL::END);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 block(PL::THREADS);
    const dim3 grid((p.nx + TX - 1) / TX, (p.ny + PL::RC - 1) / PL::RC);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = p.f2d ? PL::END : PL::END_NOF;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fine_sweep_kernel<T, LV, TL, RCT, RYT>, m.w, m.wn, m.psi, m.f, p);
}

}  // namespace

template <typename T, int RCT>
cudaError_t launch_rows(const FusedParams<T>& p, const FineMaps& m, int levels, cudaStream_t s) {
    switch (levels) {
        case 0: return launch_sweep<T, 0, false, RCT>(p, m, s);
        case 1: return launch_sweep<T, 1, false, RCT>(p, m, s);
        case 2: return launch_sweep<T, 2, false, RCT>(p, m, s);
        case 3: return launch_sweep<T, 3, false, RCT>(p, m, s);
        case 4: return launch_sweep<T, 4, false, RCT>(p, m, s);
        default: return cudaErrorInvalidValue;
    }
}

// 4 rows per thread (half the default): the shorter CTAs shrink the last,
// partly filled wave of a launch; l <= 2 only (a group covers whole cells)
template <typename T, int RCT>
cudaError_t launch_rows4(const FusedParams<T>& p, const FineMaps& m, int levels, cudaStream_t s) {
    switch (levels) {
        case 0: return launch_sweep<T, 0, false, RCT, 4>(p, m, s);
        case 1: return launch_sweep<T, 1, false, RCT, 4>(p, m, s);
        case 2: return launch_sweep<T, 2, false, RCT, 4>(p, m, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_fine_fused(const FusedParams<T>& p, const FineMaps& m, int levels,
                              cudaStream_t s, bool two_layer, int rows, int ry) {
    constexpr int R0 = Rows<T>::value;
    const int ry0 = levels >= 4 ? 16 : 8;
    if (two_layer) {   // l >= 1 only: the other layer's psi comes from the elliptic grid
        if (rows != R0 || ry != ry0) return cudaErrorInvalidValue;
        switch (levels) {
            case 1: return launch_sweep<T, 1, true, R0>(p, m, s);
            case 2: return launch_sweep<T, 2, true, R0>(p, m, s);
            case 3: return launch_sweep<T, 3, true, R0>(p, m, s);
            case 4: return launch_sweep<T, 4, true, R0>(p, m, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (ry == ry0) {
        if (rows == R0) return launch_rows<T, R0>(p, m, levels, s);
        if constexpr (sizeof(T) == 4) {
            if (rows == 64) return launch_rows<T, 64>(p, m, levels, s);
            if (rows == 32) return launch_rows<T, 32>(p, m, levels, s);
        }
    } else if (ry == 4) {
        if constexpr (sizeof(T) == 4) {
            if (rows == 64) return launch_rows4<T, 64>(p, m, levels, s);
            if (rows == 32) return launch_rows4<T, 32>(p, m, levels, s);
        }
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_fine_fused<float>(const FusedParams<float>&, const FineMaps&, int,
                                              cudaStream_t, bool, int, int);
template cudaError_t launch_fine_fused<double>(const FusedParams<double>&, const FineMaps&, int,
                                               cudaStream_t, bool, int, int);

template <typename T, int RCT>
cudaError_t launch_batch_rows(const FineMember<T>* fm, const int4* tiles, int ntiles, int levels,
                              bool forcing_field, bool pdl, cudaStream_t s) {
    switch (levels) {
        case 0: return launch_batch<T, 0, RCT>(fm, tiles, ntiles, forcing_field, pdl, s);
        case 1: return launch_batch<T, 1, RCT>(fm, tiles, ntiles, forcing_field, pdl, s);
        case 2: return launch_batch<T, 2, RCT>(fm, tiles, ntiles, forcing_field, pdl, s);
        case 3: return launch_batch<T, 3, RCT>(fm, tiles, ntiles, forcing_field, pdl, s);
        case 4: return launch_batch<T, 4, RCT>(fm, tiles, ntiles, forcing_field, pdl, s);
        default: return cudaErrorInvalidValue;
    }
}

// Members' tiles are `rows` fine rows high (ensemble_tile_rows) with the
// default rows per thread.
template <typename T>
cudaError_t launch_fine_batch(const FineMember<T>* fm, const int4* tiles, int ntiles, int levels,
                              bool forcing_field, bool pdl, cudaStream_t s, int rows) {
    if (ntiles < 1) return cudaSuccess;
    if (rows == Rows<T>::value)
        return launch_batch_rows<T, Rows<T>::value>(fm, tiles, ntiles, levels, forcing_field, pdl, s);
    if constexpr (sizeof(T) == 4) {
        if (rows == 64)
            return launch_batch_rows<T, 64>(fm, tiles, ntiles, levels, forcing_field, pdl, s);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_fine_batch<float>(const FineMember<float>*, const int4*, int, int, bool,
                                              bool, cudaStream_t, int);
template cudaError_t launch_fine_batch<double>(const FineMember<double>*, const int4*, int, int,
                                               bool, bool, cudaStream_t, int);

size_t fine_tile_rows(size_t esz) { return esz == 8 ? Rows<double>::value : Rows<float>::value; }
// the tile of ensemble members' batched sweeps: 64 rows (128 threads, 5 CTAs
// per SM in FP32; the tile the step autotuner keeps for large one-layer
// basins)
int ensemble_tile_rows(size_t esz) { return 64; }
int fine_rows_per_thread(int levels) { return levels >= 4 ? 16 : 8; }
bool fine_rows_supported(size_t esz, int layers, int levels, int rows, int ry) {
    const int ry0 = fine_rows_per_thread(levels);
    if (rows == (int)fine_tile_rows(esz) && ry == ry0) return true;
    if (esz != 4 || layers != 1) return false;
    if (ry == ry0) return rows == 64 || rows == 32;
    return ry == 4 && levels <= 2 && (rows == 64 || rows == 32);
}
int fine_part_period_x(int levels) { return TX >> levels; }
int fine_part_period_y(int levels, int rows) { return rows >> levels; }
int fine_halo_cols() { return SWX; }
int fine_block_cols() { return TX; }

QG_BOUNDS_QUERY(bounds_site_fused)

}  // namespace qg
