// step_block.cuh -- the fused collide-and-stream step of the RC-LBM
// (arXiv 2103.02119, Sec. 4) and of its raw-moment variant (RNR-LBM, Sec. 3)
// for sm_103a, FP32 and FP64: one thread block's work.  Included by the
// translation units that instantiate the kernels (rc_step.cu,
// rc_free_step.cu, rnr_step.cu).
//
// One launch advances the whole lattice by one time step.  A thread block
// owns a segment of W = BXT * VC columns -- each of its BXT threads owns VC
// consecutive cells of a row (VC = 2: one 8-byte vector in FP32, a 16-byte
// one in FP64) -- and a band of rows, and marches through the band one row at a
// time.
//
// The scheme is a template parameter of the block's work (SCH: 0 RC-LBM,
// 1 RNR-LBM, 2 chosen per lattice at run time, 3 RC-LBM without a body
// force, its force terms compiled out), so that a single-lattice kernel
// carries only its own collision; scheme -1 (no collision) is a run time
// switch of every kernel.
//
// Staging.  The populations a row pulls (plane i of the source row
// y - e_iy, columns x0-4 .. x0+W+3) are brought into shared memory by TMA
// bulk copies (cp.async.bulk, completion counted on an mbarrier), issued by
// one lane kStages rows ahead into a ring of kStages stages (four in FP32
// blocks of 128 or more threads, three otherwise).  A thread reads its
// cells' nine populations with vector shared loads (plus one scalar load for
// the planes shifted along x) and keeps them in registers until the row
// collides one iteration later, so a stage is free as soon as its row is
// read.  A cell next to a wall or a solid reads its bounced-back
// populations from global memory (with a mask, its open links still come
// from the stage), as does the first/last column of a periodic x axis
// (wrap).  Results go out as vector global stores.
//
// Iteration k:
//   1. wait for the stage of row k; load each cell's nine populations into
//      registers, sum them into its density and put it into a four-row ring
//      in shared memory (lanes of warp 0 add the density of the two columns
//      just outside the segment, one population per lane);
//   2. one barrier (which also votes on a timed-out wait);
//   3. the issuing lane refills the stage of row k with row k+3;
//   4. row k-1 collides from the populations kept in registers: its density
//      gradient comes from the ring by central differences (spacing 2 along
//      x, 2a along y; a wall or solid neighbour mirrors the cell's own
//      density), and the result is stored to the cell's slot of the output.
// The band includes one row before and after it, whose density the ring
// needs.  Even bands march up and odd bands march down, so that two
// neighbouring bands read their shared rows at about the same time.
//
// Every mbarrier wait is bounded.  A wait that runs out sets bit 0 of
// *p.status, waits (bounded again) for the block's copies still in flight,
// and the whole block returns.  A checked build (LBM_CHECKED) also tests
// every computed global, mask and shared-memory index; a failed test skips
// the access, sets bit 1 and stops the block the same way.
#pragma once
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

namespace {

// Stage ring depth: copies run kStages rows ahead.  FP32 blocks of 128 or
// more threads take four stages (76.3k against 75.1k MLUPS with three on the
// 2048 x 8192 cavity); narrower FP32 blocks and FP64 take three, where a
// fourth stage leaves room for one block fewer per SM (64-thread batch
// blocks: 9 instead of 10 per SM; the 512-lattice sweep 43.1k against 39.3k
// MLUPS with three).
template <typename T, int BXT>
__host__ __device__ constexpr int step_stages() {
    return sizeof(T) == 4 && BXT >= 128 ? 4 : 3;
}
constexpr int kHalo = 4;                // staged columns on each side of a segment
// Polls of a bounded wait: the drain of the copies in flight always uses
// kSpinLimit; the wait for a row's data uses the lattice's spin_limit (the
// same by default; a test may set it lower to make that wait run out).
constexpr unsigned kSpinLimit = kWaitPolls;

__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
    return (unsigned)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait of at most `limit` polls; false when it ran out.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          unsigned limit = kSpinLimit) {
    for (unsigned n = 0; n < limit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// N consecutive values of type T as one 4-, 8- or 16-byte access.
template <typename T, int N>
__device__ __forceinline__ void ldv(const T* p, T* out) {
    if constexpr (N * sizeof(T) == 16 && sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else if constexpr (N * sizeof(T) == 16) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        out[0] = v.x; out[1] = v.y;
    } else if constexpr (N * sizeof(T) == 8 && sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        out[0] = v.x; out[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j) out[j] = p[j];
    }
}
template <typename T, int N>
__device__ __forceinline__ void stv(T* p, const T* in) {
    if constexpr (N * sizeof(T) == 16 && sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
    } else if constexpr (N * sizeof(T) == 16) {
        *reinterpret_cast<double2*>(p) = make_double2(in[0], in[1]);
    } else if constexpr (N * sizeof(T) == 8 && sizeof(T) == 4) {
        *reinterpret_cast<float2*>(p) = make_float2(in[0], in[1]);
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j) p[j] = in[j];
    }
}

}  // namespace

template <typename T>
__host__ __device__ constexpr int step_cells_per_thread() { return 2; }

// mbarriers, the population stages, the density ring and the link-mask stages
template <typename T, int BXT>
constexpr size_t step_smem_bytes() {
    constexpr int kStages = step_stages<T, BXT>();
    constexpr int W = BXT * step_cells_per_thread<T>();
    return 128 + (size_t)kStages * 9 * (W + 2 * kHalo) * sizeof(T) + 4 * (W + 8) * sizeof(T) +
           (size_t)kStages * W;
}

// I: element-offset type, int while 9 * plane < 2^31, else long long.
__device__ __forceinline__ void mbar_inval(unsigned bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// One block's work: segment `seg` of columns and row band `band` (of nbands)
// of one lattice, from fin to fout.  smem: step_smem_bytes<T, BXT>() bytes.
// Returns false when a wait ran out (the block must stop).
// PT: KParams<T> or const KParams<T>& (a kernel parameter, or the copy in
// shared memory of a lattice of a batch).
template <typename T, bool MASK, int BXT, typename I, int SCH, typename PT = KParams<T>>
__device__ __forceinline__ bool step_block(const T* __restrict__ fin, T* __restrict__ fout,
                                           const PT p, int nbands, int seg, int band,
                                           unsigned char* smem) {
    constexpr int VC = step_cells_per_thread<T>();
    constexpr int kStages = step_stages<T, BXT>();
    constexpr int W = BXT * VC;          // segment width
    constexpr int SW = W + 2 * kHalo;    // staged row width
    constexpr int RW = W + 8;            // density ring row width
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem);
    T* stage = reinterpret_cast<T*>(smem + 128);        // [kStages][9][SW]
    T* ring = stage + kStages * 9 * SW;                 // [4][RW], column c at c - x0 + 4
    const uint8_t* smask = reinterpret_cast<const uint8_t*>(ring + 4 * RW);  // [kStages][W]
    // checked build: a failed bounds check (the access is skipped; the block
    // stops at its next vote)
    bool bad = false;
    const long long nbuf = 9 * (long long)p.plane;  // elements of a population buffer

    const int tx = threadIdx.x;
    const int lane = tx & 31;
    // the warp that issues the copies: warp 1, not warp 0, which adds the
    // halo densities (the per-row barrier waits on the slowest warp); a
    // one-warp block does both
    constexpr int kIssueWarp = BXT >= 64 ? 1 : 0;
    const int x0 = seg * W;
    const int nseg = min(W, p.nx - x0);
    const int c0 = VC * tx;              // first cell of this thread, within the segment
    const int xa = x0 + c0;              // its column
    const bool any_active = c0 < nseg;
    const bool all_active = c0 + VC <= nseg;
    const int y0 = (int)(((long long)band * p.ny) / nbands);
    const int y1 = (int)(((long long)(band + 1) * p.ny) / nbands);
    const int dir = (band & 1) ? -1 : 1;
    const int rfirst = dir > 0 ? y0 - 1 : y1;
    const int nit = (y1 - y0) + 2;
    const I pitch = p.pitch;      // row length of the link mask
    const I rs = p.rstride;       // row stride of the populations
    const I pl = (I)p.plane;

    // staged window of global columns [wstart, wend)
    const int wstart = max(x0 - kHalo, 0);
    const int wend = min(x0 + W + kHalo, p.pitch);
    const unsigned cbytes = (unsigned)((wend - wstart) * sizeof(T));
    const int dshift = wstart - (x0 - kHalo);
    const unsigned bar0 = smem_u32(bars);
    const unsigned st0 = smem_u32(stage);

    // per-thread x-wall bits: does one of my cells touch x = 0 / nx - 1?
    const bool has_first = xa == 0;
    const bool has_last = xa <= p.nx - 1 && p.nx - 1 < xa + VC;
    // a thread is on the fast path when all its cells are active, none is a
    // periodic edge column, and (per row) none has a wall or solid source
    const bool xfast = all_active && !(p.px && (has_first || has_last));

    // halo lanes of warp 0 (another warp issues the copies, so the extra
    // work is split between two warps): lanes 0..8 take population `lane` of the column
    // left of the segment, lanes 16..24 population `lane-16` of the column
    // right of it
    const int hside = lane >> 4, hi = lane & 15;
    const bool hlane = tx < 32 && hi < 9;
    const int hraw = hside == 0 ? x0 - 1 : x0 + nseg;
    int hx = hraw;
    bool hok = true;
    if (hx < 0) { if (p.px) hx += p.nx; else hok = false; }
    else if (hx >= p.nx) { if (p.px) hx -= p.nx; else hok = false; }
    const bool hpull = hlane && hok;
    if (!hok) hx = 0;
    const bool hwrap = hx != hraw || (p.px && (hx == 0 || hx == p.nx - 1));

    auto row_valid = [&](int r) { return (r >= 0 && r < p.ny) || p.py; };
    auto wrap_row = [&](int r) { return r < 0 ? r + p.ny : (r >= p.ny ? r - p.ny : r); };
    auto bits_at = [&](int cx, int rr) -> unsigned {
        if (MASK) return mask_at(p, (long long)rr * pitch + cx, bad);
        const unsigned Wb = (cx == 0) & !p.px, Eb = (cx == p.nx - 1) & !p.px;
        const unsigned S = (rr == 0) & !p.py, N = (rr == p.ny - 1) & !p.py;
        return Wb | (S << 1) | (Eb << 2) | (N << 3) | ((Wb | S) << 4) | ((Eb | S) << 5) |
               ((Eb | N) << 6) | ((Wb | N) << 7);
    };
    // link bits of my VC cells in row rr (staged in stage s); returns their
    // OR (0: all fluid, no wall)
    // Without a mask the bits split into a column part (west/east walls:
    // bits 0, 4, 7 / 2, 5, 6) and a row part (south/north walls: bits 1, 4,
    // 5 / 3, 6, 7); inactive cells are solid.
    unsigned xbits[VC];
#pragma unroll
    for (int j = 0; j < VC; ++j) {
        const int cx = xa + j;
        const unsigned Wb = (cx == 0) & !p.px, Eb = (cx == p.nx - 1) & !p.px;
        xbits[j] = (c0 + j < nseg) ? (Wb * 0x91u | Eb * 0x64u) : 0xFFu;
    }
    auto cell_bits = [&](int s, int rr, unsigned* sb) -> unsigned {
        unsigned any = 0;
        if (MASK) {
            const uint8_t* m = smask + s * W + c0;
            if constexpr (kChecked) {
                if (!idx_ok(s * W + c0, kStages * W, VC)) {
                    bad = true;
#pragma unroll
                    for (int j = 0; j < VC; ++j) sb[j] = 0xFFu;
                    return 0xFFu;
                }
            }
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                sb[j] = (c0 + j < nseg) ? (unsigned)m[j] : 0xFFu;
                any |= sb[j];
            }
        } else {
            const unsigned S = (rr == 0) & !p.py, N = (rr == p.ny - 1) & !p.py;
            const unsigned ybits = S * 0x32u | N * 0xC8u;
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                sb[j] = xbits[j] | ybits;
                any |= sb[j];
            }
        }
        return any;
    };

    // the issuing warp's lane 0: copies of the source rows of iteration k
    // into its stage, one per plane, and the row of the link mask (columns
    // x0 .. x0 + mbytes; x0 and the row pitch are multiples of 32, so the
    // copy is 16-byte aligned and stays inside the mask).  One lane issues
    // them all: every operand is then the same across the warp, so the
    // copies need no serialisation over lanes.
    const unsigned mbytes = (unsigned)min(W, p.pitch - x0);
    const unsigned sm0 = smem_u32(smask);
    auto issue = [&](int k) {
        if (lane != 0) return;
        const int s = k % kStages;
        const unsigned bar = bar0 + 8u * s;
        const int r = rfirst + dir * k;
        const bool ok = row_valid(r);
        const int rr = ok ? wrap_row(r) : 0;
        // source row of the planes with e_y = 0, +1, -1
        int srow[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            int sr = -1;
            if (ok) {
                sr = rr - (e == 0 ? 0 : (e == 1 ? 1 : -1));
                if (sr < 0 || sr >= p.ny) sr = p.py ? wrap_row(sr) : -1;
            }
            srow[e] = sr;
        }
        if constexpr (kChecked) {
            // a copy stays inside its source row and its stage row
            const bool cols_ok = wstart >= 0 && wend <= (int)rs && wstart < wend &&
                                 dshift >= 0 && dshift + (wend - wstart) <= SW;
#pragma unroll
            for (int e = 0; e < 3; ++e)
                if (srow[e] >= p.ny || (srow[e] >= 0 && !cols_ok)) {
                    bad = true;
                    srow[e] = -1;
                }
        }
        bool mcopy = MASK && ok;
        if constexpr (kChecked) {
            if (mcopy && !idx_ok((long long)rr * pitch + x0, (long long)pitch * p.ny, (int)mbytes)) {
                bad = true;
                mcopy = false;
            }
        }
        unsigned bytes = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sr = srow[ey(i) == 0 ? 0 : (ey(i) > 0 ? 1 : 2)];
            if (sr >= 0) bytes += cbytes;
        }
        if (mcopy) bytes += mbytes;
        mbar_expect_tx(bar, bytes);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sr = srow[ey(i) == 0 ? 0 : (ey(i) > 0 ? 1 : 2)];
            if (sr >= 0)
                bulk_g2s(st0 + (unsigned)(((s * 9 + i) * SW + dshift) * sizeof(T)),
                         fin + (i * pl + (I)sr * rs + wstart), cbytes, bar);
        }
        if (mcopy)
            bulk_g2s(sm0 + (unsigned)(s * W), p.lmask + ((I)rr * pitch + x0), mbytes, bar);
    };
    // (spreading the ten copies over warps 1-3 measured 5 % slower than one
    // lane of one warp issuing them all)
    const bool issuer = (tx >> 5) == kIssueWarp;

    // populations g[i][j] of my VC cells (row rr) from stage s.  Fast: vector
    // shared loads.  Otherwise cell by cell: shared loads for a fluid cell
    // without wall sources; for one next to a wall or solid, shared loads
    // for its open links and a global read of its own opposite population
    // for each blocked one (with a mask; without one the global gather of
    // all nine); the global gather of a cell on the first or last column of
    // a periodic x axis; zeros for a solid or inactive cell.
    auto load = [&](int s, int rr, const unsigned* sb, bool fast, T (*g)[VC]) {
        const T* b = stage + s * 9 * SW + (c0 + kHalo);
        if constexpr (kChecked) {
            // every stage read below lies in columns c0 + kHalo - 1 .. c0 +
            // kHalo + VC of the nine rows of stage s
            if (!(idx_ok(s * 9 * SW + c0 + kHalo - 1, kStages * 9 * SW) &&
                  idx_ok((s * 9 + 8) * SW + c0 + kHalo + VC, kStages * 9 * SW))) {
                bad = true;
#pragma unroll
                for (int i = 0; i < 9; ++i)
#pragma unroll
                    for (int j = 0; j < VC; ++j) g[i][j] = T(0);
                return;
            }
        }
        if (fast) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const T* q = b + i * SW;
                T v[VC];
                ldv<T, VC>(q, v);
                if (ex(i) == 0) {
#pragma unroll
                    for (int j = 0; j < VC; ++j) g[i][j] = v[j];
                } else if (ex(i) > 0) {  // source x - 1
                    g[i][0] = q[-1];
#pragma unroll
                    for (int j = 1; j < VC; ++j) g[i][j] = v[j - 1];
                } else {                 // source x + 1
#pragma unroll
                    for (int j = 0; j < VC - 1; ++j) g[i][j] = v[j + 1];
                    g[i][VC - 1] = q[VC];
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                const int cx = xa + j;
                T f[9];
                if (sb[j] == 0xFFu) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = T(0);
                } else if (sb[j] == 0u && !(p.px && (cx == 0 || cx == p.nx - 1))) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = b[i * SW + j - ex(i)];
                } else if (MASK && !(p.px && (cx == 0 || cx == p.nx - 1))) {
                    // With a mask (walls and solids anywhere): an open link's
                    // source is staged; a blocked one bounces back the cell's
                    // own opposite population, a global read unless the link
                    // is horizontal.  (Without a mask only the edge rows and
                    // columns come here, and the full gather measured faster.)
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (i > 0 && ((sb[j] >> (i - 1)) & 1u)) {
                            // plane opp(i) is staged at this row when e_iy = 0
                            if (ey(i) == 0)
                                f[i] = b[opp(i) * SW + j];
                            else
                                f[i] = ldg_chk(fin, opp(i) * pl + (I)rr * rs + cx, nbuf, bad);
                        } else {
                            f[i] = b[i * SW + j - ex(i)];
                        }
                    }
                } else {
                    pull(fin, p, cx, rr, sb[j], f, bad);
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i][j] = f[i];
            }
        }
    };

    if (tx == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(bar0 + 8u * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (issuer)
        for (int k = 0; k < kStages && k < nit; ++k) issue(k);

    unsigned sbp[VC];     // link bits of the previous row's cells
    bool fastp = false;   // its fast-path flag
    bool colp = false;    // whether it is collided
    int rrp = 0;          // its wrapped row index
    T dp[VC];             // its density deviations
    T gp[9][VC];          // its populations
#pragma unroll
    for (int j = 0; j < VC; ++j) { sbp[j] = 0xFFu; dp[j] = T(0); }
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j < VC; ++j) gp[i][j] = T(0);

    // With a mask the halo lanes' link bits are a global read: each row's
    // are loaded one row ahead, so that the read's latency does not sit
    // before the row barrier.
    auto halo_bits = [&](int k) -> unsigned {
        const int r = rfirst + dir * k;
        if (!(MASK && hpull && k < nit && row_valid(r))) return 0xFFu;
        return bits_at(hx, wrap_row(r));
    };
    unsigned hb_next = MASK ? halo_bits(0) : 0u;

    for (int k = 0; k < nit; ++k) {
        const int r = rfirst + dir * k;
        unsigned hb_cur = 0u;
        if constexpr (MASK) {
            hb_cur = hb_next;
            hb_next = halo_bits(k + 1);
        }
        const int s = k % kStages;
        const int slot = k & 3;
        const bool to = !mbar_wait(bar0 + 8u * s, (unsigned)((k / kStages) & 1), p.spin_limit);

        // 1. density of row r and of the two halo columns
        const bool rv = row_valid(r);
        const int rr = rv ? wrap_row(r) : 0;
        unsigned sbc[VC];
        T dc[VC];
        bool fastc = false;
        bool colc = false;
        T g[9][VC];
#pragma unroll
        for (int j = 0; j < VC; ++j) { sbc[j] = 0xFFu; dc[j] = T(0); }
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = 0; j < VC; ++j) g[i][j] = T(0);
        if (!to && rv && any_active) {
            const unsigned any = cell_bits(s, rr, sbc);
            fastc = xfast && any == 0u;
            load(s, rr, sbc, fastc, g);
            if constexpr (sizeof(T) == 4) {  // both cells in one float2
                float2 G[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) G[i] = make_float2(g[i][0], g[i][1]);
                const float2 sd = vadd(vadd(vadd(vadd(G[0], G[1]), vadd(G[2], G[3])),
                                            vadd(vadd(G[4], G[5]), vadd(G[6], G[7]))),
                                       G[8]);
                dc[0] = sd.x;
                dc[1] = sd.y;
            } else {
#pragma unroll
                for (int j = 0; j < VC; ++j)
                    dc[j] = ((g[0][j] + g[1][j]) + (g[2][j] + g[3][j])) +
                            ((g[4][j] + g[5][j]) + (g[6][j] + g[7][j])) + g[8][j];
            }
            colc = true;
        }
        if constexpr (kChecked) {
            if (!idx_ok(slot * RW + c0 + 4, 4 * RW, VC)) bad = true;
        }
        if (kChecked && bad) {
            // a checked build skips the ring row after a failed check
        } else if (all_active) {
            stv<T, VC>(ring + slot * RW + c0 + 4, dc);
        } else {  // a partial last group must not touch the right halo's slot
#pragma unroll
            for (int j = 0; j < VC; ++j)
                if (c0 + j < nseg) ring[slot * RW + c0 + 4 + j] = dc[j];
        }
        if (tx < 32) {
            T h = T(0);
            if (!to && rv && hpull) {
                const unsigned hb = MASK ? hb_cur : bits_at(hx, rr);
                if (hb != 0xFFu) {
                    const int i = hi;
                    if (hb == 0u && !hwrap) {
                        const int si = (s * 9 + i) * SW + (hx - x0 + kHalo - ex(i));
                        if (kChecked && !idx_ok(si, kStages * 9 * SW))
                            bad = true;
                        else
                            h = stage[si];
                    } else if (i > 0 && ((hb >> (i - 1)) & 1u)) {
                        h = ldg_chk(fin, opp(i) * pl + (I)rr * rs + hx, nbuf, bad);
                    } else {
                        int sx = hx - ex(i), sy = rr - ey(i);
                        sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
                        sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
                        h = ldg_chk(fin, i * pl + (I)sy * rs + sx, nbuf, bad);
                    }
                }
            }
            // offsets 1, 2, 4, 8 add the nine populations in the same order as
            // the in-thread sum above, so a density does not depend on which
            // block computes it
#pragma unroll
            for (int off = 1; off < 16; off <<= 1) h += __shfl_xor_sync(0xffffffffu, h, off);
            if (hi == 0 && hok) {
                const int ri = slot * RW + (hside == 0 ? 3 : nseg + 4);
                if (kChecked && !idx_ok(ri, 4 * RW))
                    bad = true;
                else
                    ring[ri] = h;
            }
        }

        // 2. barrier, with a vote on a timed-out wait (and, in a checked
        // build, on a failed bounds check)
        if (__syncthreads_or(to || (kChecked && bad))) {
            if (to) atomicOr(p.status, kStatusTimeout);
            if (kChecked && bad) atomicOr(p.status, kStatusBounds);
            if (tx == 0) {
                // copies issued for iterations k .. k+kStages-1 may be in flight
                for (int j = k; j < k + kStages && j < nit; ++j)
                    mbar_wait(bar0 + 8u * (j % kStages), (unsigned)((j / kStages) & 1));
            }
            return false;
        }

        // 3. refill the stage of row k (now in registers) with row k+kStages
        if (issuer && k + kStages < nit) {
            fence_proxy_async();
            issue(k + kStages);
        }

        // 4. collide the previous row
        if (k >= 2 && colp) {
            const int rc = r - dir;
            T (&gcol)[9][VC] = gp;
            const int sC = (k - 1) & 3;
            const int sN = dir > 0 ? (k & 3) : ((k - 2) & 3);
            const int sS = dir > 0 ? ((k - 2) & 3) : (k & 3);
            T dCv[VC + 2], dNv[VC], dSv[VC];
            if constexpr (kChecked) {
                // ring reads: columns c0 + 3 .. c0 + 4 + VC of rows sC, sN, sS
                if (!(idx_ok(sC * RW + c0 + 3, 4 * RW, VC + 2) &&
                      idx_ok(sN * RW + c0 + 4, 4 * RW, VC) && idx_ok(sS * RW + c0 + 4, 4 * RW, VC)))
                    bad = true;
            }
            ldv<T, VC>(ring + sC * RW + c0 + 4, dCv + 1);
            dCv[0] = ring[sC * RW + c0 + 3];
            dCv[VC + 1] = ring[sC * RW + c0 + 4 + VC];
            ldv<T, VC>(ring + sN * RW + c0 + 4, dNv);
            ldv<T, VC>(ring + sS * RW + c0 + 4, dSv);
            const bool edge_row = rc == 0 || rc == p.ny - 1;
            // density gradient by central differences; a wall or solid
            // neighbour mirrors the cell's own density
            T dxr[VC], dyr[VC], rho[VC];
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                const unsigned b = sbp[j];
                const T d = dp[j];
                const T dW = (b & 1u) ? d : dCv[j];
                const T dS = (b & 2u) ? d : dSv[j];
                const T dE = (b & 4u) ? d : dCv[j + 2];
                const T dN = (b & 8u) ? d : dNv[j];
                dxr[j] = T(0.5) * (dE - dW);
                dyr[j] = p.iah * (dN - dS);
                rho[j] = p.rho0 + d;
            }
            if (p.collide) {
                // The collision takes its constants as a copy (to_lanes).
                if constexpr (sizeof(T) == 4) {
                    // both cells in one float2 lane pair
                    static_assert(VC == 2, "FP32 collides its two cells as one float2");
                    float2 F[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) F[i] = make_float2(gcol[i][0], gcol[i][1]);
                    const float2 D = make_float2(dp[0], dp[1]);
                    const float2 Gx = make_float2(dxr[0], dxr[1]), Gy = make_float2(dyr[0], dyr[1]);
                    const float2 R = (SCH == 1 || (SCH == 2 && p.raw))
                                         ? collide_raw<float>(to_lanes(p.cc), F, D, Gx, Gy)
                                         : collide<float, SCH != 3>(to_lanes(p.cc), F, D, Gx, Gy);
                    rho[0] = R.x;
                    rho[1] = R.y;
                    // A solid cell keeps its zeros.  Without a mask the only
                    // such cells are the inactive columns past nx, stored
                    // into the row padding, which nothing reads (no fluid
                    // cell pulls from it, no read-out visits it): they take
                    // the collision's result unselected.
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (!MASK || sbp[0] != 0xFFu) gcol[i][0] = F[i].x;
                        if (!MASK || sbp[1] != 0xFFu) gcol[i][1] = F[i].y;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < VC; ++j) {
                        if (sbp[j] == 0xFFu) continue;
                        T F[9];
#pragma unroll
                        for (int i = 0; i < 9; ++i) F[i] = gcol[i][j];
                        rho[j] = (SCH == 1 || (SCH == 2 && p.raw))
                                     ? collide_raw<T>(to_lanes(p.cc), F, dp[j], dxr[j], dyr[j])
                                     : collide<T, SCH != 3>(to_lanes(p.cc), F, dp[j], dxr[j], dyr[j]);
#pragma unroll
                        for (int i = 0; i < 9; ++i) gcol[i][j] = F[i];
                    }
                }
            }
            if (p.moving && (edge_row || has_first || has_last)) {
#pragma unroll
                for (int j = 0; j < VC; ++j) {
                    const int cx = xa + j;
                    if (sbp[j] == 0xFFu || !(cx == 0 || cx == p.nx - 1 || edge_row)) continue;
                    T f[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = gcol[i][j];
                    moving_wall(p, cx, rc, rho[j], f);
#pragma unroll
                    for (int i = 0; i < 9; ++i) gcol[i][j] = f[i];
                }
            }
            const I o = (I)rc * rs + xa;
            if constexpr (kChecked) {
                if (!(rc >= 0 && rc < p.ny && xa >= 0 && xa + VC <= (int)rs)) bad = true;
            }
            if (!(kChecked && bad)) {
#pragma unroll
                for (int i = 0; i < 9; ++i) stv<T, VC>(fout + (i * pl + o), gcol[i]);
            }
        }
#pragma unroll
        for (int j = 0; j < VC; ++j) { sbp[j] = sbc[j]; dp[j] = dc[j]; }
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = 0; j < VC; ++j) gp[i][j] = g[i][j];
        fastp = fastc;
        colp = colc;
        rrp = rr;
    }
    // every copy has been waited for: retire the mbarriers so that the shared
    // memory can hold new ones (a persistent block runs step_block again)
    __syncthreads();
    if (tx == 0)
        for (int s = 0; s < kStages; ++s) mbar_inval(bar0 + 8u * s);
    if (kChecked && bad) atomicOr(p.status, kStatusBounds);  // after the last vote
    __syncthreads();
    return true;
}

// Blocks per SM the register allocator is asked to fit: in FP32 about 100
// registers a thread (the collision plus the populations kept from the
// previous row), narrower blocks scaling with it; in FP64 three blocks of 128.
template <typename T>
constexpr int step_min_blocks(int bxt) {
    return sizeof(T) != 4 ? (bxt == 128 ? 3 : 1) : bxt == 128 ? 5 : bxt == 64 ? 10 : bxt == 32 ? 20 : 1;
}

template <typename T, bool MASK, int BXT, typename I, int SCH>
__global__ void __launch_bounds__(BXT, step_min_blocks<T>(BXT))
rc_step_kernel(const T* __restrict__ fin, T* __restrict__ fout,
               const __grid_constant__ KParams<T> p, int nbands) {
    extern __shared__ __align__(128) unsigned char smem[];
    step_block<T, MASK, BXT, I, SCH, const KParams<T>&>(fin, fout, p, nbands, blockIdx.x,
                                                   blockIdx.y, smem);
}

template <typename T, bool MASK, int BXT, typename I, int SCH>
static cudaError_t launch_one(const T* fin, T* fout, const KParams<T>& p, int nbands,
                              cudaStream_t s) {
    constexpr size_t smem = step_smem_bytes<T, BXT>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(rc_step_kernel<T, MASK, BXT, I, SCH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    constexpr int W = BXT * step_cells_per_thread<T>();
    dim3 grid((p.nx + W - 1) / W, nbands);
    rc_step_kernel<T, MASK, BXT, I, SCH><<<grid, BXT, smem, s>>>(fin, fout, p, nbands);
    return cudaGetLastError();
}

template <typename T, bool MASK, int BXT, int SCH>
static cudaError_t launch_bx(const T* fin, T* fout, const KParams<T>& p, int nbands,
                             cudaStream_t s) {
    if (9LL * p.pitch * p.ny < (1LL << 31)) return launch_one<T, MASK, BXT, int, SCH>(fin, fout, p, nbands, s);
    return launch_one<T, MASK, BXT, long long, SCH>(fin, fout, p, nbands, s);
}

template <typename T, bool MASK, int SCH>
static cudaError_t launch_mask(const T* fin, T* fout, const KParams<T>& p, int bx,
                               int nbands, cudaStream_t s) {
    switch (bx) {
    case 32: return launch_bx<T, MASK, 32, SCH>(fin, fout, p, nbands, s);
    case 64: return launch_bx<T, MASK, 64, SCH>(fin, fout, p, nbands, s);
    case 128: return launch_bx<T, MASK, 128, SCH>(fin, fout, p, nbands, s);
    case 256: return launch_bx<T, MASK, 256, SCH>(fin, fout, p, nbands, s);
    default: return cudaErrorInvalidValue;
    }
}

// One step of a single lattice with the collision of scheme SCH.
template <typename T, int SCH>
static cudaError_t launch_step_scheme(const T* fin, T* fout, const KParams<T>& p, int bx,
                                      int nbands, cudaStream_t s) {
    return p.lmask ? launch_mask<T, true, SCH>(fin, fout, p, bx, nbands, s)
                   : launch_mask<T, false, SCH>(fin, fout, p, bx, nbands, s);
}

}  // namespace lbm
