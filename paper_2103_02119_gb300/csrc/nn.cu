// nn.cu -- the warm-start surrogate of include/lbm_nn.h: a 3x3-convolution
// encoder-decoder trained and evaluated on the GPU.
//
// The three GEMMs of a convolution run on the fifth-generation tensor cores
// (tcgen05.mma, kind::f16: BF16 operands from shared memory, FP32
// accumulator in tensor memory) as implicit GEMMs over NHWC activations with
// channels padded to a multiple of 8:
//   forward      M = pixels, N = cout, K = 9 cin:
//                A[p][(tap, ci)] = in(p + s(tap))[ci], B[co][(tap, ci)] = W
//   input grad   M = pixels, N = cin, K = 9 cout:
//                A[q][(tap, co)] = g(q - s(tap))[co], B[ci][(tap, co)] = W
//   weight grad  M = 9 cin, N = cout, K = pixels (split over blocks, the
//                partial sums added in a fixed order), transposed so that the
//                taps and input channels fill the 128 rows of the MMA:
//                A[(tap, ci)][p] = in(p + s(tap))[ci], B[co][p] = g(p)[co]
// with s(tap) = (dy - 1, dx - 1) and zeros outside the grid.  A CTA of 128
// threads computes a 128 x N tile (N = 16 .. 256): the threads gather K
// chunks of 64 into two shared-memory buffers in the tensor core's K-major
// core-matrix layout, one thread issues the MMAs of a chunk and commits them
// to the buffer's mbarrier, and each warp reads its 32 rows of the
// accumulator back with tcgen05.ld.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "lbm_nn.h"
#include "dev_alloc.h"
#include "nvtx_range.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kThreads = 256;
constexpr int kSplitPixels = 4096;  // pixels per block of the weight-gradient GEMM

// Division by a divisor fixed at launch, for dividends in [0, 2^31):
// q = (n m) >> s with m = ceil(2^s / d), s = 31 + ceil(log2 d) (exact in that
// range: the error of m / 2^s is below 2^-31 / d).
struct FastDiv {
    unsigned d = 1;
    unsigned long long m = 1ull << 31;
    int s = 31;
    FastDiv() = default;
    explicit FastDiv(unsigned dv) : d(dv) {
        int l = 0;
        while ((1ull << l) < dv) ++l;
        s = 31 + l;
        m = ((1ull << s) + dv - 1) / dv;
    }
    __device__ __forceinline__ unsigned div(unsigned n) const {
        return (unsigned)(((unsigned long long)n * m) >> s);
    }
};

struct Geo {
    int n, h, w;          // batch and grid
    long long P;          // pixels n h w (below 2^31: checked at creation)
    FastDiv fhw, fw;      // by h w and by w
};

Geo make_geo(int n, int h, int w, long long P) {
    Geo g;
    g.n = n;
    g.h = h;
    g.w = w;
    g.P = P;
    g.fhw = FastDiv((unsigned)(h * w));
    g.fw = FastDiv((unsigned)w);
    return g;
}

__device__ __forceinline__ bool shifted(const Geo& g, long long p, int dy, int dx, long long& q) {
    const unsigned pp = (unsigned)p;
    const unsigned nn = g.fhw.div(pp);
    const unsigned rem = pp - nn * g.fhw.d;
    const unsigned yy = g.fw.div(rem);
    const int y = (int)yy + dy, x = (int)(rem - yy * g.fw.d) + dx;
    if (y < 0 || y >= g.h || x < 0 || x >= g.w) return false;
    q = ((long long)nn * g.h + y) * g.w + x;
    return true;
}

// ---- operand tiles of the tensor-core GEMM ----
//
// A tile holds rows r (UM = 128 of A, BN of B) and the K chunk [k0, k0 + UK)
// in the tensor core's no-swizzle core-matrix layout: core matrices of
// 8 x 16 bytes stored contiguously (128 bytes), the core matrices of one
// group of 8 rows adjacent along K (leading byte offset 128) and the row
// groups 8 core matrices apart (stride byte offset 1024).  K-major: a core
// matrix row is 8 consecutive k of one row; MN-major: 8 consecutive rows at
// one k.  Every operand arrives in 16-byte pieces of one of those two kinds,
// copied by cp.async (zero-filled outside the operand).
constexpr int UM = 128, UK = 64, kGemmThreads = 128;
constexpr unsigned kLBO = 128, kSBO = (UK / 8) * 128;

// byte offset of the 16-byte piece holding rows r .. r+7 at k (MN-major) or
// row r at k .. k+7 (K-major), within a tile
__device__ __forceinline__ unsigned kmajor_off(int r, int kc) {
    return (unsigned)(r >> 3) * kSBO + (unsigned)(kc >> 3) * kLBO + (unsigned)(r & 7) * 16;
}
__device__ __forceinline__ unsigned mnmajor_off(int r8, int kc) {
    return (unsigned)(r8 >> 3) * kSBO + (unsigned)(kc >> 3) * kLBO + (unsigned)(kc & 7) * 16;
}
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
// 16 bytes global -> shared, or 16 zero bytes when !valid
__device__ __forceinline__ void cp16(unsigned dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// Forward: out = act(conv(in) + b).  M = pixels, N = cout, K = 9 cin:
// A[p][(tap, ci)] = in(p + s(tap))[ci], B[co][(tap, ci)] = W; both K-major.
struct FwdOp {
    static constexpr bool kAmn = false, kBmn = false;
    Geo g;
    FastDiv fk;        // by cin (the K index's channel count)
    const bf16* in;    // [P][cin]
    const bf16* wf;    // [cout][9 cin]
    const float* bias; // [cout]
    bf16* out;         // [P][cout]
    int cin, cout, relu;
    __host__ __device__ long long M() const { return g.P; }
    __host__ __device__ int N() const { return cout; }
    __host__ __device__ long long K() const { return 9LL * cin; }
    __device__ void load_a(unsigned t, long long m0, long long k0, long long kend, int tid) const {
#pragma unroll
        for (int i = 0; i < UM * UK / 8 / kGemmThreads; ++i) {
            const int v = tid + i * kGemmThreads, r = v >> 3, kc = (v & 7) * 8;
            const long long p = m0 + r, k = k0 + kc;
            const bf16* src = in;
            bool ok = false;
            if (p < g.P && k < kend) {
                const int tap = (int)fk.div((unsigned)k), ci = (int)k - tap * cin;
                long long q;
                if (shifted(g, p, tap / 3 - 1, tap % 3 - 1, q)) {
                    src = in + q * cin + ci;
                    ok = true;
                }
            }
            cp16(t + kmajor_off(r, kc), src, ok);
        }
    }
    __device__ void load_b(unsigned t, int n0, long long k0, long long kend, int tid,
                           int bn) const {
        for (int v = tid; v < bn * (UK / 8); v += kGemmThreads) {
            const int r = v >> 3, kc = (v & 7) * 8;
            const long long k = k0 + kc;
            const bool ok = n0 + r < cout && k < kend;
            cp16(t + kmajor_off(r, kc), ok ? wf + (long long)(n0 + r) * K() + k : wf, ok);
        }
    }
    __device__ void store16(long long row, int col0, const float* v, int) const {
        if (row >= g.P) return;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const int col = col0 + j;
            if (col >= cout) break;
            float v0 = v[j] + bias[col], v1 = v[j + 1] + bias[col + 1];
            if (relu) {
                v0 = fmaxf(v0, 0.0f);
                v1 = fmaxf(v1, 0.0f);
            }
            *reinterpret_cast<__nv_bfloat162*>(out + row * cout + col) =
                __floats2bfloat162_rn(v0, v1);
        }
    }
};

// Input gradient: gin = conv^T(gpre).  M = pixels, N = cin, K = 9 cout:
// A[q][(tap, co)] = g(q - s(tap))[co], B[ci][(tap, co)] = W; both K-major.
struct DgradOp {
    static constexpr bool kAmn = false, kBmn = false;
    Geo g;
    FastDiv fk;        // by cout
    const bf16* gpre;  // [P][cout]
    const bf16* wd;    // [cin][9 cout]
    bf16* gin;         // [P][cin]
    int cin, cout;
    __host__ __device__ long long M() const { return g.P; }
    __host__ __device__ int N() const { return cin; }
    __host__ __device__ long long K() const { return 9LL * cout; }
    __device__ void load_a(unsigned t, long long m0, long long k0, long long kend, int tid) const {
#pragma unroll
        for (int i = 0; i < UM * UK / 8 / kGemmThreads; ++i) {
            const int v = tid + i * kGemmThreads, r = v >> 3, kc = (v & 7) * 8;
            const long long p = m0 + r, k = k0 + kc;
            const bf16* src = gpre;
            bool ok = false;
            if (p < g.P && k < kend) {
                const int tap = (int)fk.div((unsigned)k), co = (int)k - tap * cout;
                long long q;
                if (shifted(g, p, 1 - tap / 3, 1 - tap % 3, q)) {
                    src = gpre + q * cout + co;
                    ok = true;
                }
            }
            cp16(t + kmajor_off(r, kc), src, ok);
        }
    }
    __device__ void load_b(unsigned t, int n0, long long k0, long long kend, int tid,
                           int bn) const {
        for (int v = tid; v < bn * (UK / 8); v += kGemmThreads) {
            const int r = v >> 3, kc = (v & 7) * 8;
            const long long k = k0 + kc;
            const bool ok = n0 + r < cin && k < kend;
            cp16(t + kmajor_off(r, kc), ok ? wd + (long long)(n0 + r) * K() + k : wd, ok);
        }
    }
    __device__ void store16(long long row, int col0, const float* v, int) const {
        if (row >= g.P) return;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const int col = col0 + j;
            if (col >= cin) break;
            *reinterpret_cast<__nv_bfloat162*>(gin + row * cin + col) =
                __floats2bfloat162_rn(v[j], v[j + 1]);
        }
    }
};

// Weight gradient, transposed so that the taps and input channels (9 cin,
// usually the larger side) fill the 128 rows: M = 9 cin, N = cout,
// K = pixels (one split of them per blockIdx.z):
// A[(tap, ci)][p] = in(p + s(tap))[ci], B[co][p] = g(p)[co], both MN-major
// (8 consecutive channels of one pixel are one 16-byte piece);
// part[z][co][(tap, ci)] = D[(tap, ci)][co].
struct WgradOp {
    static constexpr bool kAmn = true, kBmn = true;
    Geo g;
    FastDiv fk;        // by cin
    const bf16* gpre;  // [P][cout]
    const bf16* in;    // [P][cin]
    float* part;       // [splits][cout][9 cin]
    int cin, cout;
    __host__ __device__ long long M() const { return 9LL * cin; }
    __host__ __device__ int N() const { return cout; }
    __host__ __device__ long long K() const { return g.P; }
    __device__ void load_a(unsigned t, long long m0, long long k0, long long kend, int tid) const {
        // pieces (group of 8 rows, pixel): 16 x 64, consecutive threads on
        // consecutive channel groups of one pixel
#pragma unroll
        for (int i = 0; i < UM * UK / 8 / kGemmThreads; ++i) {
            const int v = tid + i * kGemmThreads, grp = v & 15, kk = v >> 4;
            const long long m = m0 + grp * 8, p = k0 + kk;
            const bf16* src = in;
            bool ok = false;
            if (m < M() && p < kend) {
                const int tap = (int)fk.div((unsigned)m), ci = (int)m - tap * cin;
                long long q;
                if (shifted(g, p, tap / 3 - 1, tap % 3 - 1, q)) {
                    src = in + q * cin + ci;
                    ok = true;
                }
            }
            cp16(t + mnmajor_off(grp * 8, kk), src, ok);
        }
    }
    __device__ void load_b(unsigned t, int n0, long long k0, long long kend, int tid,
                           int bn) const {
        for (int v = tid; v < (bn / 8) * UK; v += kGemmThreads) {
            const int grp = v % (bn / 8), kk = v / (bn / 8);
            const int co = n0 + grp * 8;
            const long long p = k0 + kk;
            const bool ok = co < cout && p < kend;
            cp16(t + mnmajor_off(grp * 8, kk), ok ? gpre + p * cout + co : gpre, ok);
        }
    }
    __device__ void store16(long long row, int col0, const float* v, int z) const {
        if (row >= M()) return;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int co = col0 + j;
            if (co >= cout) break;
            part[((long long)z * cout + co) * M() + row] = v[j];
        }
    }
};

// ---- the tensor-core GEMM: tcgen05.mma, accumulator in tensor memory ----

// shared memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), version 1 at bits 46-47, no swizzle
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// bounded wait on an mbarrier phase; false when it ran out
__device__ __forceinline__ bool mbar_wait_parity(unsigned bar, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int BN>
__host__ __device__ constexpr int tmem_cols() { return BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256; }
// pipeline depth: four stages up to 64 columns, three above (two CTAs per
// SM up to 128 columns)
template <int BN>
__host__ __device__ constexpr int gemm_stages() { return BN <= 64 ? 4 : 3; }
template <int BN>
constexpr size_t umma_smem() { return (size_t)gemm_stages<BN>() * (UM + BN) * UK * 2 + 128; }

// One CTA computes a UM x BN tile of D = A B^T over its K range, in chunks of
// UK: the threads keep NS - 1 chunks in flight as cp.async groups, one
// thread issues the four MMAs (K = 16 each) of a landed chunk and commits
// them to its stage's mbarrier, which frees the stage for the chunk NS - 1
// ahead.  The accumulator lives in BN columns of tensor memory; each warp
// reads its 32 rows back.  Every wait is bounded; one that runs out sets
// *err and the tile is not stored.
template <class Op, int BN>
__global__ void __launch_bounds__(kGemmThreads) umma_gemm_kernel(const Op op, long long kchunk,
                                                                 int* err) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
    constexpr int NS = gemm_stages<BN>();
    constexpr int TC = tmem_cols<BN>();
    constexpr unsigned kStage = (UM + BN) * UK * 2;  // A then B of one stage
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + NS * kStage);
    unsigned* tslot = reinterpret_cast<unsigned*>(bars + NS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long m0 = (long long)blockIdx.x * UM;
    const int n0 = blockIdx.y * BN;
    const long long kbeg = (long long)blockIdx.z * kchunk;
    const long long kend = min(op.K(), kbeg + kchunk);
    const int nkb = kend > kbeg ? (int)((kend - kbeg + UK - 1) / UK) : 0;
    const unsigned s0 = smem_addr(sm), bar0 = smem_addr(bars);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tslot)),
                     "n"(TC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned taddr = *tslot;
    // instruction descriptor: FP32 accumulator, BF16 A and B, their majors
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((Op::kAmn ? 1u : 0u) << 15) | ((Op::kBmn ? 1u : 0u) << 16) |
                               ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
    auto load = [&](int kb) {
        const unsigned st = s0 + (unsigned)(kb % NS) * kStage;
        const long long k0 = kbeg + (long long)kb * UK;
        op.load_a(st, m0, k0, kend, tid);
        op.load_b(st + UM * UK * 2, n0, k0, kend, tid, BN);
    };
#pragma unroll
    for (int kb = 0; kb < NS - 1; ++kb) {
        if (kb < nkb) load(kb);
        cp_commit();
    }
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % NS;
        cp_wait<NS - 2>();  // this thread's pieces of chunk kb have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();    // everyone's have
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = s0 + (unsigned)st * kStage, b0 = a0 + UM * UK * 2;
#pragma unroll
            for (int kk = 0; kk < UK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 2 * kLBO, kLBO, kSBO);
                const uint64_t bd = smem_desc(b0 + kk * 2 * kLBO, kLBO, kSBO);
                const unsigned acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar0 + 8u * st)
                : "memory");
        }
        // the chunk NS - 1 ahead goes into the stage of chunk kb - 1, once
        // the MMAs that read it are done
        const int nk = kb + NS - 1;
        if (nk < nkb) {
            if (kb >= 1) {
                const int ps = (kb - 1) % NS;
                ok &= mbar_wait_parity(bar0 + 8u * ps, (unsigned)(((kb - 1) / NS) & 1));
            }
            load(nk);
        }
        cp_commit();
    }
    // the last commit tracks every MMA of the tile
    if (nkb > 0)
        ok &= mbar_wait_parity(bar0 + 8u * ((nkb - 1) % NS), (unsigned)(((nkb - 1) / NS) & 1));
    cp_wait<0>();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const long long row = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + ((unsigned)(32 * warp) << 16) + (unsigned)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = nkb > 0 ? __uint_as_float(r[j]) : 0.0f;
        if (ok) op.store16(row, n0 + c0, v, (int)blockIdx.z);
    }
    if (!ok && lane == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "n"(TC)
                     : "memory");
}

template <class Op, int BN>
cudaError_t launch_umma_bn(const Op& op, long long kchunk, int splits, int* err,
                           cudaStream_t s) {
    constexpr size_t smem = umma_smem<BN>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(umma_gemm_kernel<Op, BN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const long long gm = (op.M() + UM - 1) / UM;
    const int gn = (op.N() + BN - 1) / BN;
    if (gm > 0x7fffffffLL) return cudaErrorInvalidValue;
    umma_gemm_kernel<Op, BN><<<dim3((unsigned)gm, gn, splits), kGemmThreads, smem, s>>>(op, kchunk,
                                                                                        err);
    return cudaGetLastError();
}

// The tile width: the smallest UMMA N (16, 32, 64, 128, 256) that covers N,
// 256 above.
#ifndef LBM_GEMM_WIDE
#define LBM_GEMM_WIDE 1
#endif
template <class Op>
cudaError_t launch_gemm(const Op& op, long long kchunk, int splits, int* err, cudaStream_t s) {
    const int n = op.N();
    if (n <= 16) return launch_umma_bn<Op, 16>(op, kchunk, splits, err, s);
    if (n <= 32) return launch_umma_bn<Op, 32>(op, kchunk, splits, err, s);
    if (n <= 64) return launch_umma_bn<Op, 64>(op, kchunk, splits, err, s);
    if (n <= 128 || !LBM_GEMM_WIDE) return launch_umma_bn<Op, 128>(op, kchunk, splits, err, s);
    return launch_umma_bn<Op, 256>(op, kchunk, splits, err, s);
}

// ---- elementwise and reduction kernels ----

__global__ void relu_mask_kernel(const bf16* out, const bf16* g, bf16* gpre, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        gpre[i] = __bfloat162float(out[i]) > 0.0f ? g[i] : __float2bfloat16_rn(0.0f);
}

// 2x2 average: (((x00 + x10) + x01) + x11) / 4, rounded once.
__global__ void pool_kernel(const bf16* in, bf16* out, int n, int h, int w, int c) {
    const int ho = h / 2, wo = w / 2;
    const long long total = (long long)n * ho * wo * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int x = (int)(r % wo);
        r /= wo;
        const int y = (int)(r % ho);
        const int nn = (int)(r / ho);
        auto at = [&](int yy, int xx) {
            return __bfloat162float(in[(((long long)nn * h + yy) * w + xx) * c + ch]);
        };
        const float s = ((at(2 * y, 2 * x) + at(2 * y + 1, 2 * x)) + at(2 * y, 2 * x + 1)) +
                        at(2 * y + 1, 2 * x + 1);
        out[i] = __float2bfloat16_rn(0.25f * s);
    }
}

// gin(2y+a, 2x+b) = 0.25 g(y, x) + gin(2y+a, 2x+b) (the skip gradient already there)
__global__ void pool_back_kernel(const bf16* g, bf16* gin, int n, int h, int w, int c,
                                 int accumulate) {
    const long long total = (long long)n * h * w * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int x = (int)(r % w);
        r /= w;
        const int y = (int)(r % h);
        const int nn = (int)(r / h);
        const float v =
            0.25f * __bfloat162float(g[(((long long)nn * (h / 2) + y / 2) * (w / 2) + x / 2) * c + ch]);
        gin[i] = __float2bfloat16_rn(accumulate ? v + __bfloat162float(gin[i]) : v);
    }
}

__global__ void up_kernel(const bf16* in, bf16* out, int n, int h, int w, int c) {
    // out is (n, 2h, 2w, c)
    const long long total = (long long)n * 4 * h * w * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int x = (int)(r % (2 * w));
        r /= 2 * w;
        const int y = (int)(r % (2 * h));
        const int nn = (int)(r / (2 * h));
        out[i] = in[(((long long)nn * h + y / 2) * w + x / 2) * c + ch];
    }
}

// gin(y, x) = ((g(2y,2x) + g(2y+1,2x)) + g(2y,2x+1)) + g(2y+1,2x+1), rounded once
__global__ void up_back_kernel(const bf16* g, bf16* gin, int n, int h, int w, int c) {
    const long long total = (long long)n * h * w * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % c);
        long long r = i / c;
        const int x = (int)(r % w);
        r /= w;
        const int y = (int)(r % h);
        const int nn = (int)(r / h);
        auto at = [&](int yy, int xx) {
            return __bfloat162float(g[(((long long)nn * 2 * h + yy) * 2 * w + xx) * c + ch]);
        };
        gin[i] = __float2bfloat16_rn(((at(2 * y, 2 * x) + at(2 * y + 1, 2 * x)) +
                                      at(2 * y, 2 * x + 1)) + at(2 * y + 1, 2 * x + 1));
    }
}

__global__ void add_kernel(const bf16* a, const bf16* b, bf16* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// host float inputs (n, h, w, 4) -> bf16 (n, h, w, 8) with zero channels 4..7
__global__ void pack_input_kernel(const float* x, bf16* out, long long pixels, int cin, int cp) {
    const long long total = pixels * cp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i % cp);
        const long long p = i / cp;
        out[i] = __float2bfloat16_rn(ch < cin ? x[p * cin + ch] : 0.0f);
    }
}

template <typename V>
__device__ __forceinline__ V block_sum(V v) {
    __shared__ V sh[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    V s = V(0);
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += sh[i];
    return s;  // valid in thread 0
}

// ---- the fixed output stage: masked smoothing and the staggered projection ----
//
// smooth:    out(p) = fl(p) sum_{dy,dx} w(dy) w(dx) fl(q) in(q), q = p + (dy, dx)
//            inside the grid, w = (1/4, 1/2, 1/4); fl from input channel 0
// unstagger: channel 1 minus its projection on (-1)^x, channel 2 minus its
//            projection on (-1)^y, over the fluid cells of each instance
// Both are self-adjoint: the backward pass applies unstagger, then smooth.

// Fluid flags: the network input's channel 0 (the solid flag) below 1/2, or
// a byte per cell (nonzero: fluid).
struct FluidIn {
    const bf16* x;
    int cp;
    __device__ __forceinline__ bool operator()(long long p) const {
        return __bfloat162float(x[p * cp]) < 0.5f;
    }
};
struct FluidBytes {
    const uint8_t* m;
    __device__ __forceinline__ bool operator()(long long p) const { return m[p] != 0; }
};

// in: bf16 [P][icp] or float [P][3]; out: float [P][3] or bf16 [P][ocp] (the
// channels past 3 zeroed)
template <bool IN_BF16, bool OUT_BF16, typename FL>
__global__ void out_smooth_kernel(const void* in, int icp, FL fluid, void* out, int ocp, int n,
                                  int h, int w) {
    const long long P = (long long)n * h * w;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % w);
        const long long r = p / w;
        const int y = (int)(r % h);
        const long long base = r / h * h;
        float acc[3] = {0.0f, 0.0f, 0.0f};
        if (fluid(p)) {
            for (int dy = -1; dy <= 1; ++dy) {
                const int yy = y + dy;
                if (yy < 0 || yy >= h) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = x + dx;
                    if (xx < 0 || xx >= w) continue;
                    const long long q = (base + yy) * w + xx;
                    if (!fluid(q)) continue;
                    const float wt = (dy == 0 ? 0.5f : 0.25f) * (dx == 0 ? 0.5f : 0.25f);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float v = IN_BF16
                                            ? __bfloat162float(static_cast<const bf16*>(in)[q * icp + c])
                                            : static_cast<const float*>(in)[q * 3 + c];
                        acc[c] = fmaf(wt, v, acc[c]);
                    }
                }
            }
        }
        if (OUT_BF16) {
            bf16* o = static_cast<bf16*>(out) + p * ocp;
            for (int c = 0; c < ocp; ++c) o[c] = __float2bfloat16_rn(c < 3 ? acc[c] : 0.0f);
        } else {
            float* o = static_cast<float*>(out) + p * 3;
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = acc[c];
        }
    }
}

// Block k: sums over the fluid cells of instance k of (-1)^x v1, (-1)^y v2 and
// the cell count, in a fixed order.
template <typename FL>
__global__ void __launch_bounds__(kThreads) stagger_sum_kernel(const float* v, FL fluid,
                                                               double* sums, int h, int w) {
    const long long hw = (long long)h * w, p0 = (long long)blockIdx.x * hw;
    double s1 = 0.0, s2 = 0.0, nf = 0.0;
    for (long long i = threadIdx.x; i < hw; i += blockDim.x) {
        const long long p = p0 + i;
        if (!fluid(p)) continue;
        const int x = (int)(i % w), y = (int)(i / w);
        s1 += (x & 1) ? -(double)v[p * 3 + 1] : (double)v[p * 3 + 1];
        s2 += (y & 1) ? -(double)v[p * 3 + 2] : (double)v[p * 3 + 2];
        nf += 1.0;
    }
    s1 = block_sum(s1);
    s2 = block_sum(s2);
    nf = block_sum(nf);
    if (threadIdx.x == 0) {
        sums[3 * blockIdx.x] = s1;
        sums[3 * blockIdx.x + 1] = s2;
        sums[3 * blockIdx.x + 2] = nf;
    }
}

template <typename FL>
__global__ void stagger_apply_kernel(const float* v, FL fluid, const double* sums, float* out,
                                     long long P, int h, int w) {
    const long long hw = (long long)h * w;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        const long long k = p / hw, i = p - k * hw;
        const int x = (int)(i % w), y = (int)(i / w);
        float o1 = v[p * 3 + 1], o2 = v[p * 3 + 2];
        const double nf = sums[3 * k + 2];
        if (nf > 0.0 && fluid(p)) {
            const float c1 = (float)(sums[3 * k] / nf), c2 = (float)(sums[3 * k + 1] / nf);
            o1 -= (x & 1) ? -c1 : c1;
            o2 -= (y & 1) ? -c2 : c2;
        }
        out[p * 3] = v[p * 3];
        out[p * 3 + 1] = o1;
        out[p * 3 + 2] = o2;
    }
}

// Bilinear prolongation by an integer factor f of cell-centred fields:
// coarse [n][hc][wc][3] -> fine [n][hc f][wc f][3].  The centre of fine cell
// (Y, X) lies at coarse coordinates ((Y + 1/2) / f - 1/2, (X + 1/2) / f - 1/2),
// clamped to the coarse cell centres (constant beyond the outermost ones);
// solid fine cells get 0.
__global__ void prolong_kernel(const float* in, const uint8_t* fluid, float* out, int n, int hc,
                               int wc, int f) {
    const int H = hc * f, W = wc * f;
    const long long P = (long long)n * H * W;
    const float inv = 1.0f / (float)f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(p % W);
        const long long r = p / W;
        const int Y = (int)(r % H);
        const long long k = r / H;
        float* o = out + p * 3;
        if (!fluid[p]) {
            o[0] = o[1] = o[2] = 0.0f;
            continue;
        }
        const float yc = fminf(fmaxf(((float)Y + 0.5f) * inv - 0.5f, 0.0f), (float)(hc - 1));
        const float xc = fminf(fmaxf(((float)X + 0.5f) * inv - 0.5f, 0.0f), (float)(wc - 1));
        const int y0 = (int)yc, x0 = (int)xc;
        const int y1 = min(y0 + 1, hc - 1), x1 = min(x0 + 1, wc - 1);
        const float ty = yc - (float)y0, tx = xc - (float)x0;
        const float* a = in + k * hc * wc * 3;
        const float* r0 = a + (long long)y0 * wc * 3;
        const float* r1 = a + (long long)y1 * wc * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float lo = fmaf(tx, r0[x1 * 3 + c] - r0[x0 * 3 + c], r0[x0 * 3 + c]);
            const float hi = fmaf(tx, r1[x1 * 3 + c] - r1[x0 * 3 + c], r1[x0 * 3 + c]);
            o[c] = fmaf(ty, hi - lo, lo);
        }
    }
}

// Masked squared error of the network's output y (FP32 [P][3], after the
// output stage): per-block partial sums (FP64) and the output gradient
// 2 (y - t) fluid / cnt (FP32 [P][3]).
__global__ void __launch_bounds__(kThreads) loss_kernel(const float* y, const float* t,
                                                        const uint8_t* fluid, float* gy,
                                                        double* part, long long pixels,
                                                        float inv_cnt) {
    double s = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pixels;
         p += (long long)gridDim.x * blockDim.x) {
        const float m = fluid[p] ? 1.0f : 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = (y[p * 3 + c] - t[p * 3 + c]) * m;
            s += (double)d * (double)d;
            gy[p * 3 + c] = 2.0f * d * inv_cnt;
        }
    }
    const double b = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void __launch_bounds__(kThreads) sum_kernel(const double* part, int n, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    const double b = block_sum(s);
    if (threadIdx.x == 0) *out = b;
}

// bias gradient: gb[co] = sum_p gpre[p][co], one block per channel
__global__ void __launch_bounds__(kThreads) bias_grad_kernel(const bf16* gpre, float* gb,
                                                             long long pixels, int cout) {
    const int co = blockIdx.x;
    float s = 0.0f;
    for (long long p = threadIdx.x; p < pixels; p += blockDim.x)
        s += __bfloat162float(gpre[p * cout + co]);
    const float b = block_sum(s);
    if (threadIdx.x == 0) gb[co] = b;
}

// dW = sum over the splits in order
__global__ void split_sum_kernel(const float* part, float* gw, int splits, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + i];
        gw[i] = s;
    }
}

// Adam on FP32 masters; counts t from 1.
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, long long n,
                            float lr, float b1, float b2, float c1, float c2, float eps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of the weights: wf[co][tap][ci] and wd[ci][tap][co] from the
// master wm[co][tap][ci]
__global__ void weight_copies_kernel(const float* wm, bf16* wf, bf16* wd, int cin, int cout) {
    const long long n = 9LL * cin * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin);
        const long long r = i / cin;
        const int tap = (int)(r % 9);
        const int co = (int)(r / 9);
        const bf16 v = __float2bfloat16_rn(wm[i]);
        wf[i] = v;
        wd[((long long)ci * 9 + tap) * cout + co] = v;
    }
}

int grid_of(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct lbm_nn {
    struct Tensor {
        int h, w, c, cp;   // grid, logical and padded channels
        bf16* v = nullptr; // activation
        bf16* g = nullptr; // its gradient
    };
    struct Conv {
        int in, out, relu;
        int cin, cout, cinp, coutp;
        float *wm, *bm, *gw, *gb, *mw, *vw, *mb, *vb;  // [coutp][9][cinp], [coutp]
        bf16 *wf, *wd;
    };
    enum Kind { CONV, POOL, UP, ADD };
    struct Op {
        Kind k;
        int a, b, out;  // tensor ids (CONV: conv index in a)
    };
    int L = 0, nb = 0, H = 0, W = 0;
    std::vector<int> ch;
    std::vector<Tensor> t;
    std::vector<Conv> conv;
    std::vector<Op> ops;
    int x_id = 0, y_id = 0;
    cudaStream_t stream = nullptr;
    float* pbuf = nullptr;     // all FP32 parameter-sized arrays
    size_t pfloats = 0;
    bf16* wbuf = nullptr;      // BF16 weight copies
    unsigned char* abuf = nullptr;  // activations and gradients
    bf16* scratch = nullptr;   // relu-masked gradient
    float* part = nullptr;     // weight-gradient split partials
    size_t part_floats = 0;
    double* dpart = nullptr;   // loss partials (+1 for the total)
    float* xin = nullptr;      // staging of host inputs (float)
    float* tgt = nullptr;
    uint8_t* fl = nullptr;
    float* yout = nullptr;     // the network's output after the output stage [P][3]
    float* gout = nullptr;     // the loss gradient of yout [P][3]
    float* tmp3 = nullptr;     // the output stage's intermediate [P][3]
    double* ssum = nullptr;    // per instance: the staggered sums and fluid count
    float* fine = nullptr;     // lbm_nn_prolong: two fine fields [max_batch][H f][W f][3]
    uint8_t* fine_fl = nullptr;  // and their fluid flags
    long long fine_cells = 0;  // cells per fine field the buffers hold
    int* gemm_err = nullptr;   // set by a GEMM whose bounded wait ran out
    long long adam_t = 0;
    int64_t launches = 0;
    char err[512] = {0};
};

namespace {

thread_local char g_nn_err[512] = "no error";

void nn_err(lbm_nn* nn, const char* fmt, ...) {
    char* dst = nn ? nn->err : g_nn_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
}

#define NCK(nn, call, what)                                                    \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            nn_err(nn, "%s: %s", what, cudaGetErrorString(e_));                \
            return e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA; \
        }                                                                      \
    } while (0)

int pad8(int c) { return (c + 7) / 8 * 8; }

long long pixels(const lbm_nn* nn, int id, int n) {
    return (long long)n * nn->t[id].h * nn->t[id].w;
}

int add_tensor(lbm_nn* nn, int h, int w, int c) {
    lbm_nn::Tensor T;
    T.h = h;
    T.w = w;
    T.c = c;
    T.cp = pad8(c);
    nn->t.push_back(T);
    return (int)nn->t.size() - 1;
}

int add_conv(lbm_nn* nn, int in, int cout, int relu) {
    const lbm_nn::Tensor X = nn->t[in];  // a copy: add_tensor grows nn->t
    const int out = add_tensor(nn, X.h, X.w, cout);
    lbm_nn::Conv c{};
    c.in = in;
    c.out = out;
    c.relu = relu;
    c.cin = X.c;
    c.cout = cout;
    c.cinp = X.cp;
    c.coutp = pad8(cout);
    nn->conv.push_back(c);
    nn->ops.push_back({lbm_nn::CONV, (int)nn->conv.size() - 1, 0, out});
    return out;
}

// Builds the network graph (see include/lbm_nn.h).
void build_graph(lbm_nn* nn) {
    nn->x_id = add_tensor(nn, nn->H, nn->W, 4);
    int x = nn->x_id;
    std::vector<int> e(nn->L);
    int h = nn->H, w = nn->W;
    for (int l = 0; l < nn->L; ++l) {
        x = add_conv(nn, x, nn->ch[l], 1);
        x = add_conv(nn, x, nn->ch[l], 1);
        e[l] = x;
        if (l < nn->L - 1) {
            h /= 2;
            w /= 2;
            const int p = add_tensor(nn, h, w, nn->ch[l]);
            nn->ops.push_back({lbm_nn::POOL, x, 0, p});
            x = p;
        }
    }
    for (int l = nn->L - 2; l >= 0; --l) {
        h *= 2;
        w *= 2;
        const int u = add_tensor(nn, h, w, nn->ch[l + 1]);
        nn->ops.push_back({lbm_nn::UP, x, 0, u});
        const int c = add_conv(nn, u, nn->ch[l], 1);
        const int s = add_tensor(nn, h, w, nn->ch[l]);
        nn->ops.push_back({lbm_nn::ADD, c, e[l], s});
        x = add_conv(nn, s, nn->ch[l], 1);
    }
    nn->y_id = add_conv(nn, x, 3, 0);
}

size_t conv_wsize(const lbm_nn::Conv& c) { return 9ull * c.cinp * c.coutp; }

lbm_status sync_weights(lbm_nn* nn) {
    for (auto& c : nn->conv) {
        weight_copies_kernel<<<grid_of((long long)conv_wsize(c)), kThreads, 0, nn->stream>>>(
            c.wm, c.wf, c.wd, c.cinp, c.coutp);
        NCK(nn, cudaGetLastError(), "weight copies");
        ++nn->launches;
    }
    return LBM_OK;
}

lbm_status upload_inputs(lbm_nn* nn, const float* x, const float* tgt, const uint8_t* fluid,
                         int n) {
    const long long P = (long long)n * nn->H * nn->W;
    NCK(nn, cudaMemcpyAsync(nn->xin, x, P * 4 * sizeof(float), cudaMemcpyHostToDevice, nn->stream),
        "cudaMemcpyAsync(H2D)");
    if (tgt)
        NCK(nn, cudaMemcpyAsync(nn->tgt, tgt, P * 3 * sizeof(float), cudaMemcpyHostToDevice,
                                nn->stream),
            "cudaMemcpyAsync(H2D)");
    if (fluid)
        NCK(nn, cudaMemcpyAsync(nn->fl, fluid, P, cudaMemcpyHostToDevice, nn->stream),
            "cudaMemcpyAsync(H2D)");
    const lbm_nn::Tensor& X = nn->t[nn->x_id];
    pack_input_kernel<<<grid_of(P * X.cp), kThreads, 0, nn->stream>>>(nn->xin, X.v, P, 4, X.cp);
    NCK(nn, cudaGetLastError(), "input packing");
    ++nn->launches;
    return LBM_OK;
}

// out = the staggered projection of v (FP32 [P][3] each), per instance.
lbm_status unstagger(lbm_nn* nn, int n, const float* v, float* out) {
    const lbm_nn::Tensor& X = nn->t[nn->x_id];
    const long long P = pixels(nn, nn->x_id, n);
    const FluidIn fl{X.v, X.cp};
    stagger_sum_kernel<<<n, kThreads, 0, nn->stream>>>(v, fl, nn->ssum, X.h, X.w);
    NCK(nn, cudaGetLastError(), "staggered sums");
    stagger_apply_kernel<<<grid_of(P), kThreads, 0, nn->stream>>>(v, fl, nn->ssum, out, P, X.h,
                                                                  X.w);
    NCK(nn, cudaGetLastError(), "staggered projection");
    nn->launches += 3;  // with the smoothing launched beside it
    return LBM_OK;
}

lbm_status forward(lbm_nn* nn, int n) {
    const cudaStream_t s = nn->stream;
    for (const auto& op : nn->ops) {
        cudaError_t e = cudaSuccess;
        if (op.k == lbm_nn::CONV) {
            const lbm_nn::Conv& c = nn->conv[op.a];
            const lbm_nn::Tensor& X = nn->t[c.in];
            FwdOp f;
            f.g = make_geo(n, X.h, X.w, pixels(nn, c.in, n));
            f.fk = FastDiv((unsigned)c.cinp);
            f.in = X.v;
            f.wf = c.wf;
            f.bias = c.bm;
            f.out = nn->t[c.out].v;
            f.cin = c.cinp;
            f.cout = c.coutp;
            f.relu = c.relu;
            e = launch_gemm(f, f.K(), 1, nn->gemm_err, s);
        } else if (op.k == lbm_nn::POOL) {
            const lbm_nn::Tensor& X = nn->t[op.a];
            pool_kernel<<<grid_of(pixels(nn, op.out, n) * X.cp), kThreads, 0, s>>>(
                X.v, nn->t[op.out].v, n, X.h, X.w, X.cp);
            e = cudaGetLastError();
        } else if (op.k == lbm_nn::UP) {
            const lbm_nn::Tensor& X = nn->t[op.a];
            up_kernel<<<grid_of(pixels(nn, op.out, n) * X.cp), kThreads, 0, s>>>(
                X.v, nn->t[op.out].v, n, X.h, X.w, X.cp);
            e = cudaGetLastError();
        } else {
            const long long cnt = pixels(nn, op.out, n) * nn->t[op.out].cp;
            add_kernel<<<grid_of(cnt), kThreads, 0, s>>>(nn->t[op.a].v, nn->t[op.b].v,
                                                         nn->t[op.out].v, cnt);
            e = cudaGetLastError();
        }
        NCK(nn, e, "forward kernels");
        ++nn->launches;
    }
    // the fixed output stage: yout = unstagger(smooth(y))
    const lbm_nn::Tensor& X = nn->t[nn->x_id];
    const lbm_nn::Tensor& Y = nn->t[nn->y_id];
    const long long P = pixels(nn, nn->y_id, n);
    out_smooth_kernel<true, false><<<grid_of(P), kThreads, 0, s>>>(
        Y.v, Y.cp, FluidIn{X.v, X.cp}, nn->tmp3, 3, n, Y.h, Y.w);
    NCK(nn, cudaGetLastError(), "output smoothing");
    return unstagger(nn, n, nn->tmp3, nn->yout);
}

// Loss of the batch (synchronous) and, through the backward pass, the
// gradients of every convolution's parameters (c.gw, c.gb).
lbm_status backward(lbm_nn* nn, int n, float* loss) {
    const cudaStream_t s = nn->stream;
    const long long P = (long long)n * nn->H * nn->W;
    std::vector<uint8_t> host_fl(P);
    NCK(nn, cudaMemcpyAsync(host_fl.data(), nn->fl, P, cudaMemcpyDeviceToHost, s),
        "cudaMemcpyAsync(D2H)");
    NCK(nn, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    long long nf = 0;
    for (long long i = 0; i < P; ++i) nf += host_fl[i] != 0;
    const float inv_cnt = nf > 0 ? (float)(1.0 / (3.0 * (double)nf)) : 0.0f;
    std::vector<bf16*> G(nn->t.size());
    for (size_t i = 0; i < nn->t.size(); ++i) G[i] = nn->t[i].g;
    const lbm_nn::Tensor& X = nn->t[nn->x_id];
    const lbm_nn::Tensor& Y = nn->t[nn->y_id];
    const int lb = grid_of(P) < 1024 ? grid_of(P) : 1024;
    loss_kernel<<<lb, kThreads, 0, s>>>(nn->yout, nn->tgt, nn->fl, nn->gout, nn->dpart, P,
                                        inv_cnt);
    NCK(nn, cudaGetLastError(), "loss kernel");
    sum_kernel<<<1, kThreads, 0, s>>>(nn->dpart, lb, nn->dpart + 1024);
    NCK(nn, cudaGetLastError(), "loss sum");
    nn->launches += 2;
    // the output stage backward: unstagger, then smooth into the gradient of
    // the last convolution's output (BF16, padded channels zeroed)
    if (lbm_status st = unstagger(nn, n, nn->gout, nn->tmp3); st != LBM_OK) return st;
    out_smooth_kernel<false, true><<<grid_of(P), kThreads, 0, s>>>(nn->tmp3, 3, FluidIn{X.v, X.cp},
                                                                   G[nn->y_id], Y.cp, n, Y.h, Y.w);
    NCK(nn, cudaGetLastError(), "output smoothing (backward)");
    std::vector<char> pool_seen(nn->t.size(), 0);
    for (int i = (int)nn->ops.size() - 1; i >= 0; --i) {
        const lbm_nn::Op& op = nn->ops[i];
        cudaError_t e = cudaSuccess;
        if (op.k == lbm_nn::CONV) {
            const lbm_nn::Conv& c = nn->conv[op.a];
            const lbm_nn::Tensor& X = nn->t[c.in];
            const lbm_nn::Tensor& O = nn->t[c.out];
            const long long Pc = pixels(nn, c.in, n);
            const bf16* gpre = G[c.out];
            if (c.relu) {
                relu_mask_kernel<<<grid_of(Pc * O.cp), kThreads, 0, s>>>(O.v, G[c.out], nn->scratch,
                                                                         Pc * O.cp);
                if ((e = cudaGetLastError()) != cudaSuccess) break;
                ++nn->launches;
                gpre = nn->scratch;
            }
            // weight gradient, split over pixels
            const int splits = (int)((Pc + kSplitPixels - 1) / kSplitPixels);
            WgradOp wg;
            wg.g = make_geo(n, X.h, X.w, Pc);
            wg.fk = FastDiv((unsigned)c.cinp);
            wg.gpre = gpre;
            wg.in = X.v;
            wg.part = nn->part;
            wg.cin = c.cinp;
            wg.cout = c.coutp;
            if ((e = launch_gemm(wg, kSplitPixels, splits, nn->gemm_err, s)) != cudaSuccess) break;
            const long long nw = (long long)conv_wsize(c);
            split_sum_kernel<<<grid_of(nw), kThreads, 0, s>>>(nn->part, c.gw, splits, nw);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            bias_grad_kernel<<<c.coutp, kThreads, 0, s>>>(gpre, c.gb, Pc, c.coutp);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            nn->launches += 3;
            if (c.in != nn->x_id) {
                DgradOp dg;
                dg.g = wg.g;
                dg.fk = FastDiv((unsigned)c.coutp);
                dg.gpre = gpre;
                dg.wd = c.wd;
                dg.gin = G[c.in];
                dg.cin = c.cinp;
                dg.cout = c.coutp;
                if ((e = launch_gemm(dg, dg.K(), 1, nn->gemm_err, s)) != cudaSuccess) break;
                ++nn->launches;
            }
        } else if (op.k == lbm_nn::POOL) {
            const lbm_nn::Tensor& X = nn->t[op.a];
            // the skip addition of the decoder has set the gradient of op.a
            pool_back_kernel<<<grid_of(pixels(nn, op.a, n) * X.cp), kThreads, 0, s>>>(
                G[op.out], G[op.a], n, X.h, X.w, X.cp, 1);
            e = cudaGetLastError();
            ++nn->launches;
        } else if (op.k == lbm_nn::UP) {
            const lbm_nn::Tensor& X = nn->t[op.a];
            up_back_kernel<<<grid_of(pixels(nn, op.a, n) * X.cp), kThreads, 0, s>>>(
                G[op.out], G[op.a], n, X.h, X.w, X.cp);
            e = cudaGetLastError();
            ++nn->launches;
        } else {
            // an addition passes its gradient to both inputs
            G[op.a] = G[op.out];
            G[op.b] = G[op.out];
        }
        if (e != cudaSuccess) {
            nn_err(nn, "backward kernels: %s", cudaGetErrorString(e));
            return LBM_ERR_CUDA;
        }
    }
    double l = 0.0;
    NCK(nn, cudaMemcpyAsync(&l, nn->dpart + 1024, sizeof(double), cudaMemcpyDeviceToHost, s),
        "cudaMemcpyAsync(D2H)");
    NCK(nn, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (loss) *loss = (float)(l * (double)inv_cnt);
    return LBM_OK;
}

// After a synchronisation: a GEMM whose bounded wait ran out leaves its word
// set (its tile was not stored).
lbm_status check_gemm(lbm_nn* nn) {
    int e = 0;
    NCK(nn, cudaMemcpy(&e, nn->gemm_err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy(D2H)");
    if (e) {
        NCK(nn, cudaMemset(nn->gemm_err, 0, sizeof(int)), "cudaMemset");
        nn_err(nn, "a tensor-core GEMM gave up waiting for its MMAs");
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

bool bad_batch(lbm_nn* nn, int n) {
    if (n < 1 || n > nn->nb) {
        nn_err(nn, "batch size %d outside [1, %d]", n, nn->nb);
        return true;
    }
    return false;
}

}  // namespace

extern "C" {

lbm_status lbm_nn_create(int levels, const int* channels, int max_batch, int height, int width,
                         uint64_t seed, void* cuda_stream, lbm_nn** out) {
    LBM_RANGE("lbm_nn_create");
    if (!out) {
        nn_err(nullptr, "out is NULL");
        return LBM_ERR_INVALID;
    }
    *out = nullptr;
    if (levels < 1 || levels > 6 || !channels || max_batch < 1 || height < 1 || width < 1 ||
        height > 4096 || width > 4096 || height % (1 << (levels - 1)) ||
        width % (1 << (levels - 1))) {
        nn_err(nullptr, "invalid network shape (levels 1..6, height and width multiples of "
                        "2^(levels-1), at most 4096)");
        return LBM_ERR_INVALID;
    }
    for (int l = 0; l < levels; ++l)
        if (channels[l] < 1 || channels[l] > 512) {
            nn_err(nullptr, "channels must lie in [1, 512]");
            return LBM_ERR_INVALID;
        }
    if ((double)max_batch * height * width > 1.0e8) {
        nn_err(nullptr, "batch of more than 1e8 cells");
        return LBM_ERR_INVALID;
    }
    lbm_nn* nn = new (std::nothrow) lbm_nn();
    if (!nn) {
        nn_err(nullptr, "host allocation failed");
        return LBM_ERR_OOM;
    }
    nn->L = levels;
    nn->ch.assign(channels, channels + levels);
    nn->nb = max_batch;
    nn->H = height;
    nn->W = width;
    nn->stream = (cudaStream_t)cuda_stream;
    build_graph(nn);
    auto fail = [&](lbm_status s) {
        std::snprintf(g_nn_err, sizeof(g_nn_err), "%s", nn->err);
        lbm_nn_destroy(nn);
        return s;
    };
#define NCKC(call, what)                                                        \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            nn_err(nn, "%s: %s", what, cudaGetErrorString(e_));                 \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA); \
        }                                                                       \
    } while (0)
    // parameters: 8 FP32 arrays per convolution (w, b, gw, gb, mw, vw, mb, vb)
    size_t pf = 0, wb = 0, maxw = 0;
    for (auto& c : nn->conv) {
        pf += 4 * (conv_wsize(c) + c.coutp);
        wb += 2 * conv_wsize(c);
        maxw = conv_wsize(c) > maxw ? conv_wsize(c) : maxw;
    }
    nn->pfloats = pf;
    NCKC(lbm::dev_alloc(&nn->pbuf, pf * sizeof(float)), "cudaMalloc(parameters)");
    NCKC(cudaMemsetAsync(nn->pbuf, 0, pf * sizeof(float), nn->stream), "cudaMemset");
    NCKC(lbm::dev_alloc(&nn->wbuf, wb * sizeof(bf16)), "cudaMalloc(weights)");
    {
        float* q = nn->pbuf;
        bf16* r = nn->wbuf;
        for (auto& c : nn->conv) {
            const size_t w = conv_wsize(c), b = c.coutp;
            c.wm = q; q += w;
            c.gw = q; q += w;
            c.mw = q; q += w;
            c.vw = q; q += w;
            c.bm = q; q += b;
            c.gb = q; q += b;
            c.mb = q; q += b;
            c.vb = q; q += b;
            c.wf = r; r += w;
            c.wd = r; r += w;
        }
    }
    // activations and their gradients, 256-byte aligned parts
    size_t ab = 0, maxt = 0;
    for (auto& T : nn->t) {
        const size_t e = (size_t)nn->nb * T.h * T.w * T.cp;
        ab += 2 * ((e * sizeof(bf16) + 255) / 256 * 256);
        maxt = e > maxt ? e : maxt;
    }
    NCKC(lbm::dev_alloc(&nn->abuf, ab), "cudaMalloc(activations)");
    NCKC(cudaMemsetAsync(nn->abuf, 0, ab, nn->stream), "cudaMemset");
    {
        unsigned char* q = nn->abuf;
        for (auto& T : nn->t) {
            const size_t e = ((size_t)nn->nb * T.h * T.w * T.cp * sizeof(bf16) + 255) / 256 * 256;
            T.v = reinterpret_cast<bf16*>(q);
            q += e;
            T.g = reinterpret_cast<bf16*>(q);
            q += e;
        }
    }
    NCKC(lbm::dev_alloc(&nn->scratch, maxt * sizeof(bf16)), "cudaMalloc(scratch)");
    const long long Pmax = (long long)nn->nb * nn->H * nn->W;
    const long long splits = (Pmax + kSplitPixels - 1) / kSplitPixels;
    nn->part_floats = (size_t)splits * maxw;
    NCKC(lbm::dev_alloc(&nn->part, nn->part_floats * sizeof(float)), "cudaMalloc(partials)");
    NCKC(lbm::dev_alloc(&nn->dpart, 1025 * sizeof(double)), "cudaMalloc(loss)");
    NCKC(lbm::dev_alloc(&nn->xin, Pmax * 4 * sizeof(float)), "cudaMalloc(inputs)");
    NCKC(lbm::dev_alloc(&nn->tgt, Pmax * 3 * sizeof(float)), "cudaMalloc(targets)");
    NCKC(lbm::dev_alloc(&nn->fl, Pmax), "cudaMalloc(fluid)");
    NCKC(lbm::dev_alloc(&nn->yout, Pmax * 3 * sizeof(float)), "cudaMalloc(outputs)");
    NCKC(lbm::dev_alloc(&nn->gout, Pmax * 3 * sizeof(float)), "cudaMalloc(output gradient)");
    NCKC(lbm::dev_alloc(&nn->tmp3, Pmax * 3 * sizeof(float)), "cudaMalloc(output stage)");
    NCKC(lbm::dev_alloc(&nn->ssum, (size_t)nn->nb * 3 * sizeof(double)), "cudaMalloc(output sums)");
    NCKC(lbm::dev_alloc(&nn->gemm_err, sizeof(int)), "cudaMalloc(error word)");
    NCKC(cudaMemsetAsync(nn->gemm_err, 0, sizeof(int), nn->stream), "cudaMemset");
#undef NCKC
    // He-normal initial weights (host generator), zero biases
    std::vector<float> params(lbm_nn_param_count(nn));
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> N01(0.0, 1.0);
    size_t k = 0;
    for (auto& c : nn->conv) {
        const double sd = std::sqrt(2.0 / (9.0 * c.cin));
        for (size_t i = 0; i < 9ull * c.cin * c.cout; ++i) params[k++] = (float)(sd * N01(rng));
        for (int i = 0; i < c.cout; ++i) params[k++] = 0.0f;
    }
    lbm_status st = lbm_nn_set_params(nn, params.data());
    if (st != LBM_OK) return fail(st);
    *out = nn;
    return LBM_OK;
}

void lbm_nn_destroy(lbm_nn* nn) {
    if (!nn) return;
    cudaFree(nn->pbuf);
    cudaFree(nn->wbuf);
    cudaFree(nn->abuf);
    cudaFree(nn->scratch);
    cudaFree(nn->part);
    cudaFree(nn->dpart);
    cudaFree(nn->xin);
    cudaFree(nn->tgt);
    cudaFree(nn->fl);
    cudaFree(nn->yout);
    cudaFree(nn->gout);
    cudaFree(nn->tmp3);
    cudaFree(nn->ssum);
    cudaFree(nn->gemm_err);
    cudaFree(nn->fine);
    cudaFree(nn->fine_fl);
    delete nn;
}

size_t lbm_nn_param_count(const lbm_nn* nn) {
    if (!nn) return 0;
    size_t n = 0;
    for (auto& c : nn->conv) n += 9ull * c.cin * c.cout + c.cout;
    return n;
}

// Host parameter vector (dy, dx, cin, cout per convolution, then biases) <->
// device masters [coutp][tap][cinp].
static lbm_status transfer_params(lbm_nn* nn, float* host, bool to_device, bool grads) {
    for (auto& c : nn->conv) {
        const size_t w = conv_wsize(c);
        std::vector<float> dev(w + c.coutp, 0.0f);
        float* dw = grads ? c.gw : c.wm;
        float* db = grads ? c.gb : c.bm;
        if (!to_device) {
            NCK(nn, cudaMemcpyAsync(dev.data(), dw, w * sizeof(float), cudaMemcpyDeviceToHost,
                                    nn->stream),
                "cudaMemcpyAsync(D2H)");
            NCK(nn, cudaMemcpyAsync(dev.data() + w, db, c.coutp * sizeof(float),
                                    cudaMemcpyDeviceToHost, nn->stream),
                "cudaMemcpyAsync(D2H)");
            NCK(nn, cudaStreamSynchronize(nn->stream), "cudaStreamSynchronize");
        }
        for (int tap = 0; tap < 9; ++tap)
            for (int ci = 0; ci < c.cin; ++ci)
                for (int co = 0; co < c.cout; ++co) {
                    float& h = host[((size_t)tap * c.cin + ci) * c.cout + co];
                    float& d = dev[((size_t)co * 9 + tap) * c.cinp + ci];
                    if (to_device) d = h;
                    else h = d;
                }
        host += 9ull * c.cin * c.cout;
        for (int co = 0; co < c.cout; ++co) {
            if (to_device) dev[w + co] = host[co];
            else host[co] = dev[w + co];
        }
        host += c.cout;
        if (to_device) {
            NCK(nn, cudaMemcpyAsync(dw, dev.data(), w * sizeof(float), cudaMemcpyHostToDevice,
                                    nn->stream),
                "cudaMemcpyAsync(H2D)");
            NCK(nn, cudaMemcpyAsync(db, dev.data() + w, c.coutp * sizeof(float),
                                    cudaMemcpyHostToDevice, nn->stream),
                "cudaMemcpyAsync(H2D)");
            NCK(nn, cudaStreamSynchronize(nn->stream), "cudaStreamSynchronize");
        }
    }
    return LBM_OK;
}

lbm_status lbm_nn_get_params(lbm_nn* nn, float* params) {
    if (!nn || !params) return LBM_ERR_INVALID;
    return transfer_params(nn, params, false, false);
}

lbm_status lbm_nn_set_params(lbm_nn* nn, const float* params) {
    if (!nn || !params) return LBM_ERR_INVALID;
    lbm_status s = transfer_params(nn, const_cast<float*>(params), true, false);
    if (s != LBM_OK) return s;
    for (auto& c : nn->conv) {
        const size_t w = conv_wsize(c);
        NCK(nn, cudaMemsetAsync(c.mw, 0, w * sizeof(float), nn->stream), "cudaMemset");
        NCK(nn, cudaMemsetAsync(c.vw, 0, w * sizeof(float), nn->stream), "cudaMemset");
        NCK(nn, cudaMemsetAsync(c.mb, 0, c.coutp * sizeof(float), nn->stream), "cudaMemset");
        NCK(nn, cudaMemsetAsync(c.vb, 0, c.coutp * sizeof(float), nn->stream), "cudaMemset");
    }
    nn->adam_t = 0;
    s = sync_weights(nn);
    if (s != LBM_OK) return s;
    NCK(nn, cudaStreamSynchronize(nn->stream), "cudaStreamSynchronize");
    return LBM_OK;
}

lbm_status lbm_nn_forward(lbm_nn* nn, const float* x, int n, float* y) {
    LBM_RANGE("lbm_nn_forward");
    if (!nn || !x || !y) return LBM_ERR_INVALID;
    if (bad_batch(nn, n)) return LBM_ERR_INVALID;
    lbm_status s = upload_inputs(nn, x, nullptr, nullptr, n);
    if (s == LBM_OK) s = forward(nn, n);
    if (s != LBM_OK) return s;
    const long long P = (long long)n * nn->H * nn->W;
    NCK(nn, cudaMemcpyAsync(y, nn->yout, P * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                            nn->stream),
        "cudaMemcpyAsync(D2H)");
    NCK(nn, cudaStreamSynchronize(nn->stream), "cudaStreamSynchronize");
    return check_gemm(nn);
}

lbm_status lbm_nn_prolong(lbm_nn* nn, const float* y, int n, int factor, const uint8_t* fluid,
                          float* out) {
    LBM_RANGE("lbm_nn_prolong");
    if (!nn || !y || !fluid || !out) return LBM_ERR_INVALID;
    if (bad_batch(nn, n)) return LBM_ERR_INVALID;
    if (factor < 1 || factor > 16) {
        nn_err(nn, "factor %d outside [1, 16]", factor);
        return LBM_ERR_INVALID;
    }
    const int H = nn->H * factor, W = nn->W * factor;
    const long long cells = (long long)H * W;
    const cudaStream_t s = nn->stream;
    if (cells > nn->fine_cells) {
        // grown on demand, kept until the network is destroyed
        NCK(nn, cudaStreamSynchronize(s), "cudaStreamSynchronize");
        cudaFree(nn->fine);
        cudaFree(nn->fine_fl);
        nn->fine = nullptr;
        nn->fine_fl = nullptr;
        nn->fine_cells = 0;
        NCK(nn, lbm::dev_alloc(&nn->fine, 2 * (size_t)nn->nb * cells * 3 * sizeof(float)),
            "cudaMalloc(fine fields)");
        NCK(nn, lbm::dev_alloc(&nn->fine_fl, (size_t)nn->nb * cells), "cudaMalloc(fine fluid)");
        nn->fine_cells = cells;
    }
    const long long Pc = (long long)n * nn->H * nn->W, P = (long long)n * cells;
    float* f0 = nn->fine;
    float* f1 = nn->fine + (size_t)nn->nb * cells * 3;
    // the coarse fields go through the output stage's buffer, free between calls
    NCK(nn, cudaMemcpyAsync(nn->tmp3, y, Pc * 3 * sizeof(float), cudaMemcpyHostToDevice, s),
        "cudaMemcpyAsync(H2D)");
    NCK(nn, cudaMemcpyAsync(nn->fine_fl, fluid, P, cudaMemcpyHostToDevice, s),
        "cudaMemcpyAsync(H2D)");
    const FluidBytes fl{nn->fine_fl};
    prolong_kernel<<<grid_of(P), kThreads, 0, s>>>(nn->tmp3, nn->fine_fl, f0, n, nn->H, nn->W,
                                                   factor);
    NCK(nn, cudaGetLastError(), "prolongation");
    out_smooth_kernel<false, false><<<grid_of(P), kThreads, 0, s>>>(f0, 3, fl, f1, 3, n, H, W);
    NCK(nn, cudaGetLastError(), "output smoothing (fine)");
    stagger_sum_kernel<<<n, kThreads, 0, s>>>(f1, fl, nn->ssum, H, W);
    NCK(nn, cudaGetLastError(), "staggered sums (fine)");
    stagger_apply_kernel<<<grid_of(P), kThreads, 0, s>>>(f1, fl, nn->ssum, f0, P, H, W);
    NCK(nn, cudaGetLastError(), "staggered projection (fine)");
    nn->launches += 4;
    NCK(nn, cudaMemcpyAsync(out, f0, P * 3 * sizeof(float), cudaMemcpyDeviceToHost, s),
        "cudaMemcpyAsync(D2H)");
    NCK(nn, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return LBM_OK;
}

lbm_status lbm_nn_gradients(lbm_nn* nn, const float* x, const float* target,
                            const uint8_t* fluid, int n, float* loss, float* grads) {
    LBM_RANGE("lbm_nn_gradients");
    if (!nn || !x || !target || !fluid) return LBM_ERR_INVALID;
    if (bad_batch(nn, n)) return LBM_ERR_INVALID;
    lbm_status s = upload_inputs(nn, x, target, fluid, n);
    if (s == LBM_OK) s = forward(nn, n);
    if (s == LBM_OK) s = backward(nn, n, loss);
    if (s == LBM_OK) s = check_gemm(nn);
    if (s == LBM_OK && grads) s = transfer_params(nn, grads, false, true);
    return s;
}

lbm_status lbm_nn_train_step(lbm_nn* nn, const float* x, const float* target,
                             const uint8_t* fluid, int n, float lr, float* loss) {
    LBM_RANGE("lbm_nn_train_step");
    if (!nn || !x || !target || !fluid) return LBM_ERR_INVALID;
    if (bad_batch(nn, n)) return LBM_ERR_INVALID;
    if (!(lr > 0.0f) || !std::isfinite(lr)) {
        nn_err(nn, "learning rate must be finite and > 0");
        return LBM_ERR_INVALID;
    }
    lbm_status s = upload_inputs(nn, x, target, fluid, n);
    if (s == LBM_OK) s = forward(nn, n);
    if (s == LBM_OK) s = backward(nn, n, loss);
    if (s != LBM_OK) return s;
    ++nn->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)nn->adam_t);
    const float c2 = 1.0f - (float)std::pow(0.999, (double)nn->adam_t);
    for (auto& c : nn->conv) {
        const long long w = (long long)conv_wsize(c);
        adam_kernel<<<grid_of(w), kThreads, 0, nn->stream>>>(c.wm, c.gw, c.mw, c.vw, w, lr, b1, b2,
                                                             c1, c2, 1e-8f);
        NCK(nn, cudaGetLastError(), "adam");
        adam_kernel<<<grid_of(c.coutp), kThreads, 0, nn->stream>>>(c.bm, c.gb, c.mb, c.vb, c.coutp,
                                                                   lr, b1, b2, c1, c2, 1e-8f);
        NCK(nn, cudaGetLastError(), "adam");
        nn->launches += 2;
    }
    s = sync_weights(nn);
    if (s != LBM_OK) return s;
    NCK(nn, cudaStreamSynchronize(nn->stream), "cudaStreamSynchronize");
    return check_gemm(nn);
}

int64_t lbm_nn_launch_count(const lbm_nn* nn) { return nn ? nn->launches : -1; }

const char* lbm_nn_last_error(const lbm_nn* nn) { return nn ? nn->err : g_nn_err; }

}  // extern "C"
