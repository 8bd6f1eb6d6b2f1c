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
// Tile: 128 rows x 64 complex columns (MMA M = 128, N = 128), K in chunks
// of 16 complex (32 real).  Shared-memory operands use the canonical K-major
// no-swizzle layout (core matrix 8 rows x 16 bytes; LBO = distance between
// K-adjacent core matrices = 128 rows x 16 B, SBO = distance between 8-row
// groups = 128 B).  A arrives by TMA already in that order (FP32; TF32 uses
// it as is, BF16x3 splits it into hi/lo planes); B columns are gathered per
// instance and expanded into the real 2x2 form.  One thread issues the MMAs
// into an FP32 accumulator in TMEM (two 128-column accumulators), read back
// with tcgen05.ld for the epilogue (power-of-two scale, scattered complex64
// stores through the output bit positions, max-|x| tracking).
//
// Every mbarrier wait is bounded; on timeout the kernel records an error
// code in *err, skips the remaining work, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace tnk {

namespace {

constexpr int TBM = 128;      // rows per tile (MMA M, TMEM lanes)
constexpr int TBN = 64;       // complex columns per tile
constexpr int TBNR = 2 * TBN; // real columns (MMA N)
constexpr int TBK = 16;       // complex k per chunk
constexpr int TBKR = 2 * TBK; // real k per chunk
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

// byte offset of element (row, kr) in a K-major no-swizzle tile of 128 rows,
// element size es bytes
__device__ __forceinline__ uint32_t kmaj_off(int row, int kr, int es) {
    const int kb = kr * es;
    return uint32_t((kb >> 4) * (TBM * 16) + (row >> 3) * 128 + (row & 7) * 16 + (kb & 15));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait(int pending) {
    switch (pending) {
        case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
        case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
    }
}

__device__ __forceinline__ void named_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// 4-D TMA tile load (shared::cluster destination = this CTA's own memory),
// completing on an mbarrier with a byte count.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Persistent warp-specialised kernel.
//   warp 17    : lane 0 streams A: one TMA tile load per chunk (128 rows x
//                16 complex k, already in the K-major core-matrix order)
//                into a ring of RST raw stages, several chunks ahead.
//   warps 0-7  : B columns by cp.async (LOOK chunks ahead), expanded into the
//                real 2x2 block form; BF16x3: A split into hi/lo from the
//                raw ring.  TF32 reads A straight from the raw ring.
//   warp 8     : TMEM allocation; lane 0 issues tcgen05.mma and commits.
//   warps 9-16 : epilogue, two warps per TMEM lane quadrant (warp % 4), each
//                draining 32 of the tile's 64 complex columns; two
//                accumulators so that a tile's epilogue overlaps the next
//                tile's MMAs.
constexpr int NPROD = 256;   // warps 0-7
constexpr int MMA_WARP = 8;
constexpr int EPI_WARP0 = 9; // warps 9-16: two per TMEM lane quadrant
constexpr int NEPI = 256;
constexpr int TMA_WARP = 17;
constexpr int NTHREADS = 576;
constexpr int ACC_COLS = 128;
constexpr int TMEM_COLS2 = 256;

template <int PREC>
struct Cfg {
    static constexpr int ST = PREC == 1 ? 4 : 3;      // MMA stages (B; BF16x3: also A hi/lo)
    static constexpr int RST = PREC == 1 ? 6 : 4;     // raw A stages filled by TMA
    static constexpr int BRST = 6;                    // raw B stages (per-thread cp.async pieces)
    static constexpr int LOOK = BRST - 1;             // B chunks issued ahead
    static constexpr int SLOT_RAW = TBM * TBK * 8;    // FP32 A chunk, [16-byte k column][row]
    static constexpr int SLOT_A = PREC == 2 ? TBM * TBKR * 4 : 0;
    static constexpr int SLOT_B = TBNR * TBKR * 4;
    static constexpr int SLOT_BRAW = TBN * TBK * 8;   // raw complex64 B chunk
    static constexpr int OFF_RAW = 0;
    static constexpr int OFF_A = OFF_RAW + RST * SLOT_RAW;
    static constexpr int OFF_B = OFF_A + ST * SLOT_A;
    static constexpr int OFF_BRAW = OFF_B + ST * SLOT_B;
    static constexpr int OFF_CTRL = OFF_BRAW + BRST * SLOT_BRAW;
};

struct EpiMeta {
    int64_t cbase[TBN];
    int64_t inst[TBN];
    float sc[TBN];
    int32_t eb[TBN];
    int32_t EB[TBN];
    uint32_t mx[TBN];
    int32_t ea, EA;
    int32_t mt, pad;
};

struct Ctrl {
    uint64_t full[4], empty[4], rfull[8], rempty[8], tfull[2], tempty[2];
    uint32_t tmem_base;
    int32_t abort_;
    int32_t epi_fail[2];  // epilogue-uniform abort decisions, by tile parity
    EpiMeta epi[2];
};

template <int PREC>
constexpr size_t smem_bytes() {
    return size_t(Cfg<PREC>::OFF_CTRL) + sizeof(Ctrl) + 128;
}
static_assert(smem_bytes<1>() <= 232448 && smem_bytes<2>() <= 232448, "shared memory above 227 KB");

// tile T of a step: column-tile record e = T / mtiles, row tile T % mtiles
__device__ __forceinline__ int4 tile_rec(const StepDesc &d, int64_t T, int64_t mtiles) {
    return __ldg(d.trec + T / mtiles);
}

template <int PREC>
__global__ void __launch_bounds__(NTHREADS, 1)  // 18 warps: at most 96 registers (5 warps on a sub-partition)
    k_step_gemm_tc(const StepDesc d, int64_t mtiles, int32_t *err, const __grid_constant__ CUtensorMap tmA) {
    using C = Cfg<PREC>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    Ctrl &X = *reinterpret_cast<Ctrl *>(sm + C::OFF_CTRL);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = d.n_ctab * mtiles;
    const int N = 1 << d.nb;
    const int64_t M = int64_t(1) << d.mb;
    const int K = 1 << d.kb;
    const int nch = (K + TBK - 1) / TBK;
    const int64_t my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total_chunks = my_tiles * nch;

    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&X.tmem_base)),
                     "r"(TMEM_COLS2)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < C::ST; ++s) {
            mbar_init(&X.full[s], NPROD);
            mbar_init(&X.empty[s], 1);
        }
        for (int s = 0; s < C::RST; ++s) {
            mbar_init(&X.rfull[s], 1);
            mbar_init(&X.rempty[s], PREC == 2 ? NPROD : 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&X.tfull[a], 1);
            mbar_init(&X.tempty[a], NEPI);
        }
        X.abort_ = *reinterpret_cast<volatile int32_t *>(err);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = X.tmem_base;
    volatile int32_t *abort_flag = &X.abort_;
    auto give_up = [&]() {
        atomicExch(err, 1);
        *abort_flag = 1;
    };
    auto tile_of = [&](int64_t l) { return int64_t(blockIdx.x) + l * gridDim.x; };

    if (warp == TMA_WARP) {
        // ------------------------------------------------------------ A stream
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            int64_t issued = 0;
            bool ok = true;
            for (int64_t l = 0; l < my_tiles && ok && !*abort_flag; ++l) {
                const int64_t T = tile_of(l);
                const int4 r = tile_rec(d, T, mtiles);
                const int m0 = int((T % mtiles) * TBM);
                for (int c = 0; c < nch; ++c, ++issued) {
                    const int rs = int(issued % C::RST);
                    if (!mbar_wait(&X.rempty[rs], (uint32_t(issued / C::RST) & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&X.rfull[rs], C::SLOT_RAW);
                    tma_load_4d(smem_u32(sm + C::OFF_RAW + rs * C::SLOT_RAW), &tmA, 0, m0, 8 * c, r.z, &X.rfull[rs]);
                }
            }
            if (!ok) give_up();
            // loads still in flight land before the CTA leaves (bounded)
            for (int64_t j = issued > C::RST ? issued - C::RST : 0; j < issued; ++j)
                mbar_wait(&X.rfull[j % C::RST], uint32_t(j / C::RST) & 1u);
        }
        __syncwarp();
    } else if (warp < NPROD / 32) {
        // ------------------------------------------------------------ B loads, A split
        const int bcol = tid & 63, kqb = tid >> 6;
        int64_t bbase[2] = {-1, -1};
        int64_t issued = 0;
        // metadata pipeline: records two tiles ahead, B instance one tile ahead
        int4 rec_pf[2] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
        int ib_pf = 0;
        auto col_inst = [&](const int4 &r) -> int64_t {  // instance of this thread's B column, or -1
            const int64_t gc = int64_t(r.w) + bcol;
            return gc < (int64_t(r.y) << d.nb) ? int64_t(r.x) + (gc >> d.nb) : -1;
        };
        if (my_tiles > 0) {
            rec_pf[0] = tile_rec(d, tile_of(0), mtiles);
            if (my_tiles > 1) rec_pf[1] = tile_rec(d, tile_of(1), mtiles);
            const int64_t ci = col_inst(rec_pf[0]);
            ib_pf = ci >= 0 ? __ldg(d.instab + ci).y : 0;
        }
        for (int64_t gch = 0; gch < total_chunks && !*abort_flag; ++gch) {
            // B pieces run LOOK chunks ahead.  Each thread reads back only
            // the 32 bytes it copied, and its raw slot was last used by a
            // chunk it has already expanded, so the ring needs no barrier.
            while (issued < total_chunks && issued <= gch + C::LOOK) {
                const int64_t l = issued / nch;
                const int c = int(issued - l * nch);
                const int bslot = int(issued % C::BRST);
                if (c == 0) {
                    const int4 r = rec_pf[l & 1];
                    const int64_t ci = col_inst(r);
                    // column-affine B: column n of instance ib starts at ib*sB + n*K
                    bbase[l & 1] = ci >= 0 ? int64_t(ib_pf) * d.sB + (((int64_t(r.w) + bcol) & (N - 1)) << d.kb) : -1;
                    if (l + 1 < my_tiles) {
                        const int64_t cn = col_inst(rec_pf[(l + 1) & 1]);
                        ib_pf = cn >= 0 ? __ldg(d.instab + cn).y : 0;
                    }
                    if (l + 2 < my_tiles) rec_pf[l & 1] = tile_rec(d, tile_of(l + 2), mtiles);
                }
                {  // B: this thread's column, k quad kqb
                    const int64_t bb = bbase[l & 1];
                    const uint32_t dst = smem_u32(sm + C::OFF_BRAW + bslot * C::SLOT_BRAW) + uint32_t(tid) * 32;
                    const int k = c * TBK + 4 * kqb;
                    const bool v = bb >= 0 && k + 3 < K;
                    const float2 *src = v ? d.B + bb + k : d.B;
                    cp_async16(dst, src, v ? 16 : 0);
                    cp_async16(dst + 16, v ? src + 2 : d.B, v ? 16 : 0);
                }
                cp_async_commit();
                ++issued;
            }
            const int slot = int(gch % C::ST);
            // the MMA stage is free once the MMAs of chunk gch - ST are done
            if (!mbar_wait(&X.empty[slot], (uint32_t(gch / C::ST) & 1u) ^ 1u)) {
                give_up();
                break;
            }
            if (PREC == 2) {
                // A: split the raw FP32 chunk into hi/lo (rows 8 at a time,
                // 16-byte k columns p and p+1 of the raw chunk per item)
                const int rs = int(gch % C::RST);
                if (!mbar_wait(&X.rfull[rs], uint32_t(gch / C::RST) & 1u)) {
                    give_up();
                    break;
                }
                const uint8_t *raw = sm + C::OFF_RAW + rs * C::SLOT_RAW;
                uint8_t *bh = sm + C::OFF_A + slot * C::SLOT_A, *bl = bh + TBM * TBKR * 2;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int item = tid + NPROD * j;  // 0..511
                    const int row = item & (TBM - 1), p = item >> 7;
                    const float4 v0 = *reinterpret_cast<const float4 *>(raw + (2 * p) * (TBM * 16) + row * 16);
                    const float4 v1 = *reinterpret_cast<const float4 *>(raw + (2 * p + 1) * (TBM * 16) + row * 16);
                    const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        hi[q] = __float2bfloat16_rn(x[q]);
                        lo[q] = __float2bfloat16_rn(x[q] - __bfloat162float(hi[q]));
                    }
                    *reinterpret_cast<uint4 *>(bh + kmaj_off(row, 8 * p, 2)) = *reinterpret_cast<uint4 *>(hi);
                    *reinterpret_cast<uint4 *>(bl + kmaj_off(row, 8 * p, 2)) = *reinterpret_cast<uint4 *>(lo);
                }
                mbar_arrive(&X.rempty[rs]);
            }
            cp_async_wait(int(issued - gch - 1));
            // B: expand this thread's prefetched piece into the MMA layout
            const uint8_t *braw = sm + C::OFF_BRAW + int(gch % C::BRST) * C::SLOT_BRAW + tid * 32;
            {
                const float4 p0 = *reinterpret_cast<const float4 *>(braw);
                const float4 p1 = *reinterpret_cast<const float4 *>(braw + 16);
                const float2 t4[4] = {make_float2(p0.x, p0.y), make_float2(p0.z, p0.w), make_float2(p1.x, p1.y),
                                      make_float2(p1.z, p1.w)};
                const float r0[8] = {t4[0].x, -t4[0].y, t4[1].x, -t4[1].y, t4[2].x, -t4[2].y, t4[3].x, -t4[3].y};
                const float r1[8] = {t4[0].y, t4[0].x, t4[1].y, t4[1].x, t4[2].y, t4[2].x, t4[3].y, t4[3].x};
                uint8_t *base = sm + C::OFF_B + slot * C::SLOT_B;
                if (PREC == 1) {
                    *reinterpret_cast<float4 *>(base + kmaj_off(2 * bcol, 8 * kqb, 4)) = make_float4(r0[0], r0[1], r0[2], r0[3]);
                    *reinterpret_cast<float4 *>(base + kmaj_off(2 * bcol, 8 * kqb + 4, 4)) = make_float4(r0[4], r0[5], r0[6], r0[7]);
                    *reinterpret_cast<float4 *>(base + kmaj_off(2 * bcol + 1, 8 * kqb, 4)) = make_float4(r1[0], r1[1], r1[2], r1[3]);
                    *reinterpret_cast<float4 *>(base + kmaj_off(2 * bcol + 1, 8 * kqb + 4, 4)) = make_float4(r1[4], r1[5], r1[6], r1[7]);
                } else {
                    __align__(16) __nv_bfloat16 h0[8], l0[8], h1[8], l1[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        h0[q] = __float2bfloat16_rn(r0[q]);
                        l0[q] = __float2bfloat16_rn(r0[q] - __bfloat162float(h0[q]));
                        h1[q] = __float2bfloat16_rn(r1[q]);
                        l1[q] = __float2bfloat16_rn(r1[q] - __bfloat162float(h1[q]));
                    }
                    uint8_t *blo = base + TBNR * TBKR * 2;
                    *reinterpret_cast<uint4 *>(base + kmaj_off(2 * bcol, 8 * kqb, 2)) = *reinterpret_cast<uint4 *>(h0);
                    *reinterpret_cast<uint4 *>(blo + kmaj_off(2 * bcol, 8 * kqb, 2)) = *reinterpret_cast<uint4 *>(l0);
                    *reinterpret_cast<uint4 *>(base + kmaj_off(2 * bcol + 1, 8 * kqb, 2)) = *reinterpret_cast<uint4 *>(h1);
                    *reinterpret_cast<uint4 *>(blo + kmaj_off(2 * bcol + 1, 8 * kqb, 2)) = *reinterpret_cast<uint4 *>(l1);
                }
            }
            proxy_fence();
            mbar_arrive(&X.full[slot]);
        }
        cp_async_wait(0);
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t LBO = TBM * 16, SBO = 128;
            int64_t gch = 0;
            for (int64_t l = 0; l < my_tiles && !*abort_flag; ++l) {
                const int acc = int(l & 1);
                if (!mbar_wait(&X.tempty[acc], (uint32_t(l >> 1) & 1u) ^ 1u)) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const uint32_t dtm = tmem + uint32_t(acc * ACC_COLS);
                bool ok = true;
                for (int c = 0; c < nch; ++c, ++gch) {
                    const int slot = int(gch % C::ST);
                    const int rs = int(gch % C::RST);
                    if (!mbar_wait(&X.full[slot], uint32_t(gch / C::ST) & 1u)) {
                        ok = false;
                        break;
                    }
                    if (PREC == 1 && !mbar_wait(&X.rfull[rs], uint32_t(gch / C::RST) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (PREC == 1) {
                        const uint32_t id = idesc(2u);
                        const uint32_t a0 = smem_u32(sm + C::OFF_RAW + rs * C::SLOT_RAW);
                        const uint32_t b0 = smem_u32(sm + C::OFF_B + slot * C::SLOT_B);
#pragma unroll
                        for (int j = 0; j < TBKR / 8; ++j) {
                            const uint32_t off = uint32_t(2 * j) * LBO;
                            mma_tf32(dtm, sdesc(a0 + off, LBO, SBO), sdesc(b0 + off, LBO, SBO), id,
                                     (c > 0 || j > 0) ? 1u : 0u);
                        }
                        mma_commit(&X.empty[slot]);
                        mma_commit(&X.rempty[rs]);
                    } else {
                        const uint32_t id = idesc(1u);
                        const uint32_t ah = smem_u32(sm + C::OFF_A + slot * C::SLOT_A), al = ah + TBM * TBKR * 2;
                        const uint32_t bh = smem_u32(sm + C::OFF_B + slot * C::SLOT_B), bl = bh + TBNR * TBKR * 2;
#pragma unroll
                        for (int j = 0; j < TBKR / 16; ++j) {
                            const uint32_t off = uint32_t(2 * j) * LBO;
                            mma_f16(dtm, sdesc(ah + off, LBO, SBO), sdesc(bh + off, LBO, SBO), id,
                                    (c > 0 || j > 0) ? 1u : 0u);
                            mma_f16(dtm, sdesc(ah + off, LBO, SBO), sdesc(bl + off, LBO, SBO), id, 1u);
                            mma_f16(dtm, sdesc(al + off, LBO, SBO), sdesc(bh + off, LBO, SBO), id, 1u);
                        }
                        mma_commit(&X.empty[slot]);
                    }
                }
                if (!ok) {
                    give_up();
                    break;
                }
                mma_commit(&X.tfull[acc]);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = tid - EPI_WARP0 * 32;     // 0..255
        const int lanegrp = warp & 3;           // TMEM lanes 32*lanegrp ...
        const int half = (warp - EPI_WARP0) >> 2;  // complex columns 32*half ...
        const int row = lanegrp * 32 + lane;
        // metadata of tile l into X.epi[l & 1] (threads 0..63: one column each)
        auto meta = [&](int64_t l) {
            EpiMeta &em = X.epi[l & 1];
            const int64_t T = int64_t(blockIdx.x) + l * gridDim.x;
            const int4 r = tile_rec(d, T, mtiles);
            if (e == 0) {
                em.ea = d.mxA ? exp_of(__ldg(d.mxA + r.z)) : 0;
                em.EA = __ldg(d.EA + r.z);
                em.mt = int(T % mtiles);
            }
            if (e < TBN) {
                const int64_t gc = int64_t(r.w) + e;
                em.mx[e] = 0;
                if (gc < (int64_t(r.y) << d.nb)) {
                    const int64_t inst = int64_t(r.x) + (gc >> d.nb);
                    const int ib = __ldg(d.instab + inst).y;
                    em.inst[e] = inst;
                    em.cbase[e] = inst * d.sC + dep(gc & (N - 1), d.pCn, d.nb);
                    em.eb[e] = d.mxB ? exp_of(__ldg(d.mxB + ib)) : 0;
                    em.EB[e] = __ldg(d.EB + ib);
                } else {
                    em.inst[e] = -1;
                    em.cbase[e] = -1;
                    em.eb[e] = 0;
                    em.EB[e] = 0;
                }
            }
        };
        // per-column scale 2^-(ea + eb), once the tile's exponents are in place
        auto scales = [&](int64_t l) {
            EpiMeta &em = X.epi[l & 1];
            if (e < TBN) em.sc[e] = pow2f(-(em.ea + em.eb[e]));
        };
        if (my_tiles > 0) meta(0);
        if (e == 0) X.epi_fail[0] = X.epi_fail[1] = 0;
        named_sync(1, NEPI);
        if (my_tiles > 0) scales(0);
        for (int64_t l = 0; l < my_tiles; ++l) {
            const int acc = int(l & 1);
            EpiMeta &em = X.epi[acc];
            if (l + 1 < my_tiles) meta(l + 1);  // overlaps the wait for tile l's accumulator
            const int64_t m0 = int64_t(em.mt) * TBM;
            if (!mbar_wait(&X.tfull[acc], uint32_t(l >> 1) & 1u)) atomicOr(&X.epi_fail[acc], 1);
            if (e == 0 && *abort_flag) atomicOr(&X.epi_fail[acc], 1);
            named_sync(1, NEPI);
            if (X.epi_fail[acc]) {  // uniform: read between barriers
                if (e == 0) give_up();
                break;
            }
            if (e == 0) X.epi_fail[acc ^ 1] = 0;  // next tile's slot; its last readers are done
            tc_fence_after();
            const int64_t m = m0 + row;
            const int64_t offc = m < M ? dep(m, d.pCm, d.mb) : -1;
            // this warp's 32 complex columns = 64 accumulator columns, in two
            // rounds of 16 complex columns (two x16 loads and one wait each).
            // Scaled stores, then the per-instance max-|x|: each column's
            // warp maximum lands in lane j = column, and runs of min(N, 32)
            // lanes (one instance's columns) are combined with xor-shuffles.
            // No branch depends on the column, so the loop pipelines.
            uint32_t colmax = 0;
#pragma unroll
            for (int rnd = 0; rnd < 2; ++rnd) {
                float v[32];
                {
                    const uint32_t ta = tmem + uint32_t(acc * ACC_COLS + half * 64 + rnd * 32) + (uint32_t(lanegrp * 32) << 16);
                    uint32_t r[32];
#pragma unroll
                    for (int q = 0; q < 2; ++q)
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                            : "=r"(r[16 * q + 0]), "=r"(r[16 * q + 1]), "=r"(r[16 * q + 2]), "=r"(r[16 * q + 3]),
                              "=r"(r[16 * q + 4]), "=r"(r[16 * q + 5]), "=r"(r[16 * q + 6]), "=r"(r[16 * q + 7]),
                              "=r"(r[16 * q + 8]), "=r"(r[16 * q + 9]), "=r"(r[16 * q + 10]), "=r"(r[16 * q + 11]),
                              "=r"(r[16 * q + 12]), "=r"(r[16 * q + 13]), "=r"(r[16 * q + 14]), "=r"(r[16 * q + 15])
                            : "r"(ta + uint32_t(16 * q)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = rnd * 16 + jj;
                    const int col = half * 32 + j;
                    const int64_t cb = em.cbase[col];
                    const float sc = em.sc[col];
                    const float2 o = make_float2(v[2 * jj] * sc, v[2 * jj + 1] * sc);
                    const bool ok = offc >= 0 && cb >= 0;
                    if (ok) d.C[cb + offc] = o;
                    if (d.mxC) {
                        const uint32_t mj = ok ? __float_as_uint(fmaxf(fabsf(o.x), fabsf(o.y))) : 0u;
                        const uint32_t rj = __reduce_max_sync(0xffffffffu, mj);
                        colmax = lane == j ? rj : colmax;
                    }
                }
            }
            if (d.mxC) {
                const int runlen = N < 32 ? N : 32;
                for (int sft = 1; sft < runlen; sft <<= 1) colmax = max(colmax, __shfl_xor_sync(0xffffffffu, colmax, sft));
                if ((lane & (runlen - 1)) == 0 && colmax) atomicMax(&em.mx[half * 32 + lane], colmax);
            }
            tc_fence_before();
            mbar_arrive(&X.tempty[acc]);
            named_sync(1, NEPI);
            if (e < TBN && em.inst[e] >= 0) {
                // exponent of the instance, written once (at its n = 0 column, row tile 0)
                const int64_t gc_n = em.cbase[e] - em.inst[e] * d.sC;  // dep(n) == 0 iff n == 0
                if (gc_n == 0 && em.mt == 0) d.EC[em.inst[e]] = em.EA + em.ea + em.EB[e] + em.eb[e];
                // em.mx[e] != 0 only where a run of this instance's columns
                // starts (instance start, or the second epilogue half)
                if (d.mxC && em.mx[e]) record_max(d.mxC + em.inst[e], em.mx[e]);
            }
            if (l + 1 < my_tiles) scales(l + 1);  // meta(l + 1) is visible since the last barrier
            named_sync(1, NEPI);  // em (this parity) is rewritten by meta(l + 2)
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS2) : "memory");
    }
}

}  // namespace

bool gemm_tc_supports(const StepDesc &d) {
    // K >= 8 complex (at least half a chunk), 64 <= M < 2^31 rows
    return d.kb >= 3 && d.mb >= 6 && d.mb <= 30 && d.kb <= 24;
}

namespace {
int g_num_sms = 0;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}

cudaError_t init_kernels() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", reinterpret_cast<void **>(&g_encode), 12000,
                                             cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !g_encode) return cudaErrorNotSupported;
    }
    e = cudaFuncSetAttribute(k_step_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<1>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_step_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<2>());
}

// The A operand of a step as a 4-D tensor for TMA: (4 floats = one 16-byte
// k column of a row, rows m, 16-byte k columns, instances).  The box
// (4, 128, 8, 1) lands in shared memory as [k column][row][16 bytes], the
// K-major core-matrix order the MMA descriptors use.  Rows past M and k past
// K read as zeros.
cudaError_t make_a_map(const StepDesc &d, int64_t n_inst_a, CUtensorMap *map) {
    if (!g_encode) return cudaErrorNotReady;
    const cuuint64_t K = cuuint64_t(1) << d.kb;
    const cuuint64_t dims[4] = {4, cuuint64_t(1) << d.mb, K / 2, cuuint64_t(n_inst_a)};
    const cuuint64_t strides[3] = {K * 8, 16, cuuint64_t(d.sA) * 8};
    const cuuint32_t box[4] = {4, TBM, TBKR / 4, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2 *>(d.A), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step_gemm_tc(const StepDesc &d, const CUtensorMap *a_map, int precision, int32_t *err,
                                cudaStream_t s) {
    if (!gemm_tc_supports(d)) return cudaErrorNotSupported;
    if (g_num_sms <= 0 || !a_map) return cudaErrorNotReady;  // init_kernels() / make_a_map() not called
    const int64_t M = int64_t(1) << d.mb;
    const int64_t mtiles = (M + TBM - 1) / TBM;
    const int64_t tiles = d.n_ctab * mtiles;
    if (tiles <= 0) return cudaSuccess;
    const int64_t grid = tiles < g_num_sms ? tiles : g_num_sms;
    if (precision == 1)
        k_step_gemm_tc<1><<<dim3((unsigned)grid), NTHREADS, smem_bytes<1>(), s>>>(d, mtiles, err, *a_map);
    else
        k_step_gemm_tc<2><<<dim3((unsigned)grid), NTHREADS, smem_bytes<2>(), s>>>(d, mtiles, err, *a_map);
    return cudaGetLastError();
}

}  // namespace tnk
