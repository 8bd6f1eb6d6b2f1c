// Tensor-core (tcgen05, sm_103a) grouped complex GEMM step.
//
// C[i](m, n) = sum_k A[a(i)](m, k) B[b(i)](k, n) for the output instances of
// one group (one shared A instance), as one real GEMM per CTA tile:
//
//   real k'  = 2k + c   (c = 0: Re, 1: Im)       -- A's complex row as stored
//   real col = 2n + c'  (c' = 0: Re, 1: Im)      -- C's complex row as stored
//   Bt[2n  ][2k] =  Re B(k,n)   Bt[2n  ][2k+1] = -Im B(k,n)
//   Bt[2n+1][2k] =  Im B(k,n)   Bt[2n+1][2k+1] =  Re B(k,n)
//
// so that Re C = Re A Re B - Im A Im B and Im C = Re A Im B + Im A Re B with
// 4 real multiply-adds per complex one (8 flops per complex MAC, nothing
// wasted).  Precisions:
//   TF32   : one kind::tf32 product of the FP32 operands.
//   BF16x3 : x = hi + lo with hi = bf16(x), lo = bf16(x - hi); three
//            kind::f16 products hi*hi + hi*lo + lo*hi into the same FP32
//            accumulator.
//
// CTA: 128 threads, tile BM = 128 rows x 64 complex columns (MMA M = 128,
// N = 128), K in chunks of 16 complex (32 real) through two shared-memory
// stages in the canonical K-major no-swizzle layout (core matrix 8 rows x
// 16 bytes; LBO = distance between K-adjacent core matrices = 128 rows x
// 16 B, SBO = distance between 8-row groups = 128 B).  All threads stage;
// one thread issues the MMAs and commits them to the stage's mbarrier; the
// FP32 accumulator lives in 128 TMEM columns and is read back with
// tcgen05.ld for the epilogue (power-of-two scale, scattered complex64
// stores through the output bit positions, max-|x| tracking).
//
// Every mbarrier wait is bounded; on timeout the kernel records an error
// code in *err, skips the remaining work, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace tnk {

namespace {

constexpr int TBM = 128;      // rows per tile (MMA M, TMEM lanes)
constexpr int TBN = 64;       // complex columns per tile
constexpr int TBNR = 2 * TBN; // real columns (MMA N)
constexpr int TBK = 16;       // complex k per chunk
constexpr int TBKR = 2 * TBK; // real k per chunk
constexpr int TMEM_COLS = 128;
constexpr unsigned long long WAIT_NS = 200000000ull;  // 200 ms per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ int exp_of(uint32_t bits) {
    if (bits == 0u) return 0;
    int e = int((bits >> 23) & 0xffu) - 127;
    return max(-126, min(126, e));
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ int64_t dep(int64_t x, const int8_t *pos, int nbits) {
    int64_t r = 0;
    for (int j = 0; j < nbits; ++j) r |= ((x >> j) & 1) << pos[j];
    return r;
}

__device__ __forceinline__ void record_max(uint32_t *slot, uint32_t v) {
    if (v > __ldcg(slot)) atomicMax(slot, v);
}

// shared-memory matrix descriptor: start, LBO, SBO (bytes, 16-byte units),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3fffu);
    d |= uint64_t((lbo >> 4) & 0x3fffu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3fffu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// instruction descriptor: FP32 accumulate, A/B K-major, M = 128, N = TBNR
__device__ __forceinline__ uint32_t idesc(uint32_t ab_format) {
    uint32_t d = 0;
    d |= 1u << 4;                 // D format: F32
    d |= ab_format << 7;          // A format
    d |= ab_format << 10;         // B format
    d |= uint32_t(TBNR >> 3) << 17;
    d |= uint32_t(TBM >> 4) << 24;
    return d;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait (WAIT_NS of wall clock); false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// byte offset of element (row, kr) in a K-major no-swizzle tile of 128 rows,
// element size es bytes
__device__ __forceinline__ uint32_t kmaj_off(int row, int kr, int es) {
    const int kb = kr * es;
    return uint32_t((kb >> 4) * (TBM * 16) + (row >> 3) * 128 + (row & 7) * 16 + (kb & 15));
}

struct __align__(16) Smem {
    // stage s: tf32 uses a[s] (16 KB) and b[s]; bf16 uses the halves
    // a[s] = {hi (8 KB), lo (8 KB)}, b[s] likewise
    uint8_t a[2][TBM * TBKR * 4];
    uint8_t b[2][TBNR * TBKR * 4];
    uint64_t bar[2];
    uint32_t tmem_base;
    int64_t offA[TBM];
    int64_t offC[TBM];
    int64_t bbase[TBN];
    int64_t cbase[TBN];
    int32_t eb[TBN];
    uint32_t mx[TBN];
    int64_t ia;
    int ea;
    int abort_;
};

template <int PREC>  // 1 = TF32, 2 = BF16x3
__global__ void __launch_bounds__(128) k_step_gemm_tc(const StepDesc d, int ctiles, int mtiles, int32_t *err) {
    extern __shared__ uint8_t smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t bid = blockIdx.x;
    const int mt = int(bid % mtiles);
    const int64_t rest = bid / mtiles;
    const int ct = int(rest % ctiles);
    const int64_t g = rest / ctiles;
    const int64_t i0 = d.gfirst[g];
    const int64_t icount = d.gfirst[g + 1] - i0;
    const int N = 1 << d.nb;
    const int64_t M = int64_t(1) << d.mb;
    const int K = 1 << d.kb;
    const int64_t cols = icount * N;
    const int64_t c0 = int64_t(ct) * TBN;
    if (c0 >= cols) return;  // uniform
    if (*reinterpret_cast<volatile int32_t *>(err) != 0) return;  // an earlier CTA gave up
    const int64_t m0 = int64_t(mt) * TBM;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const int64_t sig = i0 / d.nOut, beta = i0 - sig * d.nOut;
        S.ia = int64_t(d.sigA[sig]) * d.nOutA + d.outA[beta];
        S.ea = d.mxA ? exp_of(d.mxA[S.ia]) : 0;
        S.abort_ = 0;
    }
    {
        const int64_t m = m0 + tid;
        S.offA[tid] = m < M ? dep(m, d.pAm, d.mb) : -1;
        S.offC[tid] = m < M ? dep(m, d.pCm, d.mb) : -1;
    }
    if (tid < TBN) {
        const int c = tid;
        const int64_t gc = c0 + c;
        S.mx[c] = 0;
        if (gc < cols) {
            const int64_t inst = i0 + gc / N;
            const int n = int(gc % N);
            const int64_t sig = inst / d.nOut, beta = inst - sig * d.nOut;
            const int64_t ib = int64_t(d.sigB[sig]) * d.nOutB + d.outB[beta];
            S.bbase[c] = ib * d.sB + dep(n, d.pBn, d.nb);
            S.cbase[c] = inst * d.sC + dep(n, d.pCn, d.nb);
            S.eb[c] = d.mxB ? exp_of(d.mxB[ib]) : 0;
        } else {
            S.bbase[c] = -1;
            S.cbase[c] = -1;
            S.eb[c] = 0;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < TBN && S.cbase[tid] >= 0 && mt == 0) {
        const int64_t gc = c0 + tid;
        if (gc % N == 0) {
            const int64_t inst = i0 + gc / N;
            const int64_t sig = inst / d.nOut, beta = inst - sig * d.nOut;
            const int64_t ib = int64_t(d.sigB[sig]) * d.nOutB + d.outB[beta];
            d.EC[inst] = d.EA[S.ia] + S.ea + d.EB[ib] + S.eb[tid];
        }
    }
    const uint32_t tmem = S.tmem_base;
    const float2 *A = d.A + S.ia * d.sA;
    const int nchunks = (K + TBK - 1) / TBK;
    const int kc = K < TBK ? K : TBK;  // valid complex k in a chunk
    constexpr uint32_t LBO = TBM * 16, SBO = 128;
    bool ok = true;

    for (int c = 0; c < nchunks && ok; ++c) {
        const int s = c & 1;
        if (c >= 2) {
            if (!mbar_wait(&S.bar[s], uint32_t((c - 2) >> 1) & 1u)) {
                ok = false;
                break;
            }
            tc_fence_after();
        }
        const int k0 = c * TBK;
        // ---- stage A: units of 4 complex (32 B) per row; 128 rows x 4 units
        for (int u = tid; u < TBM * (TBK / 4); u += 128) {
            const int rl = u & 7, kq = (u >> 3) & 3, rh = u >> 5;
            const int row = rh * 8 + rl;
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
            if (S.offA[row] >= 0) {
                const float2 *src = A + S.offA[row] + k0 + 4 * kq;
                if (4 * kq + 3 < kc) {
                    v0 = __ldg(reinterpret_cast<const float4 *>(src));
                    v1 = __ldg(reinterpret_cast<const float4 *>(src) + 1);
                } else {
                    float2 t[4];
                    for (int j = 0; j < 4; ++j) t[j] = (4 * kq + j < kc) ? __ldg(src + j) : make_float2(0.f, 0.f);
                    v0 = make_float4(t[0].x, t[0].y, t[1].x, t[1].y);
                    v1 = make_float4(t[2].x, t[2].y, t[3].x, t[3].y);
                }
            }
            if (PREC == 1) {
                uint8_t *base = S.a[s];
                *reinterpret_cast<float4 *>(base + kmaj_off(row, 8 * kq, 4)) = v0;
                *reinterpret_cast<float4 *>(base + kmaj_off(row, 8 * kq + 4, 4)) = v1;
            } else {
                const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    hi[j] = __float2bfloat16_rn(x[j]);
                    lo[j] = __float2bfloat16_rn(x[j] - __bfloat162float(hi[j]));
                }
                uint8_t *bh = S.a[s], *bl = S.a[s] + TBM * TBKR * 2;
                *reinterpret_cast<uint4 *>(bh + kmaj_off(row, 8 * kq, 2)) = *reinterpret_cast<uint4 *>(hi);
                *reinterpret_cast<uint4 *>(bl + kmaj_off(row, 8 * kq, 2)) = *reinterpret_cast<uint4 *>(lo);
            }
        }
        // ---- stage B: 64 complex columns x 4 units of 4 complex k
        for (int u = tid; u < TBN * (TBK / 4); u += 128) {
            const int col = u % TBN, kq = u / TBN;
            float2 t[4];
            for (int j = 0; j < 4; ++j) {
                const int k = 4 * kq + j;
                t[j] = (S.bbase[col] >= 0 && k < kc) ? __ldg(d.B + S.bbase[col] + k0 + k) : make_float2(0.f, 0.f);
            }
            // row 2col: (Re, -Im) pairs; row 2col+1: (Im, Re) pairs
            const float r0[8] = {t[0].x, -t[0].y, t[1].x, -t[1].y, t[2].x, -t[2].y, t[3].x, -t[3].y};
            const float r1[8] = {t[0].y, t[0].x, t[1].y, t[1].x, t[2].y, t[2].x, t[3].y, t[3].x};
            if (PREC == 1) {
                uint8_t *base = S.b[s];
                *reinterpret_cast<float4 *>(base + kmaj_off(2 * col, 8 * kq, 4)) = make_float4(r0[0], r0[1], r0[2], r0[3]);
                *reinterpret_cast<float4 *>(base + kmaj_off(2 * col, 8 * kq + 4, 4)) = make_float4(r0[4], r0[5], r0[6], r0[7]);
                *reinterpret_cast<float4 *>(base + kmaj_off(2 * col + 1, 8 * kq, 4)) = make_float4(r1[0], r1[1], r1[2], r1[3]);
                *reinterpret_cast<float4 *>(base + kmaj_off(2 * col + 1, 8 * kq + 4, 4)) = make_float4(r1[4], r1[5], r1[6], r1[7]);
            } else {
                __nv_bfloat16 h0[8], l0[8], h1[8], l1[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    h0[j] = __float2bfloat16_rn(r0[j]);
                    l0[j] = __float2bfloat16_rn(r0[j] - __bfloat162float(h0[j]));
                    h1[j] = __float2bfloat16_rn(r1[j]);
                    l1[j] = __float2bfloat16_rn(r1[j] - __bfloat162float(h1[j]));
                }
                uint8_t *bh = S.b[s], *bl = S.b[s] + TBNR * TBKR * 2;
                *reinterpret_cast<uint4 *>(bh + kmaj_off(2 * col, 8 * kq, 2)) = *reinterpret_cast<uint4 *>(h0);
                *reinterpret_cast<uint4 *>(bl + kmaj_off(2 * col, 8 * kq, 2)) = *reinterpret_cast<uint4 *>(l0);
                *reinterpret_cast<uint4 *>(bh + kmaj_off(2 * col + 1, 8 * kq, 2)) = *reinterpret_cast<uint4 *>(h1);
                *reinterpret_cast<uint4 *>(bl + kmaj_off(2 * col + 1, 8 * kq, 2)) = *reinterpret_cast<uint4 *>(l1);
            }
        }
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            if (PREC == 1) {
                const uint32_t id = idesc(2u);
                const uint32_t a0 = smem_u32(S.a[s]), b0 = smem_u32(S.b[s]);
#pragma unroll
                for (int j = 0; j < TBKR / 8; ++j) {  // K = 8 tf32 = 2 core-matrix columns per MMA
                    const uint32_t off = uint32_t(2 * j) * LBO;
                    mma_tf32(tmem, sdesc(a0 + off, LBO, SBO), sdesc(b0 + off, LBO, SBO), id, (c > 0 || j > 0) ? 1u : 0u);
                }
            } else {
                const uint32_t id = idesc(1u);
                const uint32_t ah = smem_u32(S.a[s]), al = ah + TBM * TBKR * 2;
                const uint32_t bh = smem_u32(S.b[s]), bl = bh + TBNR * TBKR * 2;
#pragma unroll
                for (int j = 0; j < TBKR / 16; ++j) {  // K = 16 bf16 = 2 core-matrix columns per MMA
                    const uint32_t off = uint32_t(2 * j) * LBO;
                    mma_f16(tmem, sdesc(ah + off, LBO, SBO), sdesc(bh + off, LBO, SBO), id, (c > 0 || j > 0) ? 1u : 0u);
                    mma_f16(tmem, sdesc(ah + off, LBO, SBO), sdesc(bl + off, LBO, SBO), id, 1u);
                    mma_f16(tmem, sdesc(al + off, LBO, SBO), sdesc(bh + off, LBO, SBO), id, 1u);
                }
            }
            mma_commit(&S.bar[s]);
        }
    }
    // wait for the last two commits (every MMA of the tile)
    if (ok) {
        for (int c = (nchunks >= 2 ? nchunks - 2 : 0); c < nchunks; ++c)
            if (!mbar_wait(&S.bar[c & 1], uint32_t(c >> 1) & 1u)) ok = false;
    }
    if (!ok) {
        atomicExch(err, 1);
        S.abort_ = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!S.abort_) {
        const int row = warp * 32 + lane;
        const bool rv = S.offC[row] >= 0;
        const int64_t offc = S.offC[row];
#pragma unroll 1
        for (int cb = 0; cb < TBNR / 16; ++cb) {
            float v[16];
            tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(cb * 16), v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = cb * 8 + j;
                if (!rv || S.cbase[col] < 0) continue;
                const float sc = pow2f(-(S.ea + S.eb[col]));
                const float2 o = make_float2(v[2 * j] * sc, v[2 * j + 1] * sc);
                d.C[S.cbase[col] + offc] = o;
                if (d.mxC) atomicMax(&S.mx[col], __float_as_uint(fmaxf(fabsf(o.x), fabsf(o.y))));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (d.mxC && !S.abort_ && tid < TBN && S.cbase[tid] >= 0) {
        const int64_t inst = i0 + (c0 + tid) / N;
        record_max(d.mxC + inst, S.mx[tid]);
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace

bool gemm_tc_supports(const StepDesc &d) {
    // K >= 8 complex (at least half a chunk), M >= 64 rows
    return d.kb >= 3 && d.mb >= 6 && d.kb <= 24;
}

cudaError_t launch_step_gemm_tc(const StepDesc &d, int precision, int32_t *err, cudaStream_t s) {
    if (!gemm_tc_supports(d)) return cudaErrorNotSupported;
    const int64_t M = int64_t(1) << d.mb;
    const int64_t N = int64_t(1) << d.nb;
    const int64_t ctiles = (int64_t(d.max_group) * N + TBN - 1) / TBN;
    const int64_t mtiles = (M + TBM - 1) / TBM;
    const int64_t blocks = d.n_groups * ctiles * mtiles;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL || ctiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    // padded so that every descriptor-addressed read stays inside the
    // allocation even for a misread of the LBO/SBO roles
    const size_t smem = (sizeof(Smem) + 128 > 96 * 1024 ? sizeof(Smem) + 128 : 96 * 1024);
    if (precision == 1) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_step_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_step_gemm_tc<1><<<dim3((unsigned)blocks), 128, smem, s>>>(d, (int)ctiles, (int)mtiles, err);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_step_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_step_gemm_tc<2><<<dim3((unsigned)blocks), 128, smem, s>>>(d, (int)ctiles, (int)mtiles, err);
    }
    return cudaGetLastError();
}

}  // namespace tnk
