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
// of 16 complex (32 real).  A arrives by TMA as 128 rows of 128 bytes in
// the 128-byte swizzled K-major layout (TF32 uses it as is; BF16x3 splits
// it into hi and lo and keeps them in tensor memory, one row per lane, so
// that its MMAs read only B from shared memory: shared-memory bandwidth is
// what bounds the long-K steps).  B columns
// are gathered per instance, expanded into the real 2x2 form and stored in
// the K-major no-swizzle layout (core matrix 8 rows x 16 bytes; LBO =
// distance between K-adjacent core matrices = 128 rows x 16 B, SBO =
// distance between 8-row groups = 128 B): chunk by chunk beside A
// (streaming, MODE 0), once per group or column tile and kept in shared
// memory (resident, MODE 1, with the power-of-two rescale folded in), or
// every B instance of the step once per launch (dictionary, MODE 2).  One
// thread issues the MMAs into an FP32 accumulator in TMEM (two 128-column
// accumulators), read back with tcgen05.ld for the epilogue: power-of-two
// scale and max-|x| tracking, then each half tile goes through shared
// memory, reordered by C address (the output bit positions), and leaves as
// coalesced 16-byte stores.
//
// Every mbarrier wait is bounded; on timeout the kernel records an error
// code in *err, skips the remaining work, frees its TMEM and returns.
#include <algorithm>
#include <type_traits>
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

// fire-and-forget global max (a reduction, no returned value: the issuing
// thread never waits on memory)
__device__ __forceinline__ void record_max(uint32_t *slot, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(slot), "r"(v) : "memory");
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

// shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: rows of 128 bytes, 8-row atoms of 1024 bytes (SBO), the
// 16-byte units of row r XOR-permuted by r mod 8.  A K step inside the row
// starts 32 bytes further on (the swizzle is applied to the address).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    return sdesc(saddr, 16, 1024) | (uint64_t(2) << 61);
}

// instruction descriptor: FP32 accumulate, A/B K-major, M = 128, N = nreal
// (a multiple of 16, at most TBNR)
__device__ __forceinline__ uint32_t idesc(uint32_t ab_format, uint32_t nreal) {
    uint32_t d = 0;
    d |= 1u << 4;                 // D format: F32
    d |= ab_format << 7;          // A format
    d |= ab_format << 10;         // B format
    d |= (nreal >> 3) << 17;
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

// try_wait that may suspend the thread for up to `ns` nanoseconds (it
// returns as soon as the phase completes)
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// bounded wait (WAIT_NS of wall clock); false on timeout.  Waiting threads
// sleep in the barrier (suspend hint) instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait_sleep(bar, parity, 100000u))
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

// A from tensor memory (a_tm: lane 0, first column of the K step)
__device__ __forceinline__ void mma_f16_ts(uint32_t d, uint32_t a_tm, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tm), "l"(b), "r"(id), "r"(acc)
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

// byte offset of element (row, kr) in a K-major no-swizzle tile of nr rows
// (a multiple of 8), element size es bytes
__device__ __forceinline__ uint32_t kmaj_off(int row, int kr, int es, int nr = TBM) {
    const int kb = kr * es;
    return uint32_t((kb >> 4) * (nr * 16) + (row >> 3) * 128 + (row & 7) * 16 + (kb & 15));
}

// The same core matrices ordered by 8-row group first: group (row >> 3) at
// 8 TBKR es bytes, the K core matrices of a group contiguous (128 bytes
// apart).  Two such chunks of 128 rows placed back to back form one operand
// of 256 rows (a column-tile pair of two B instances).
__device__ __forceinline__ uint32_t rmaj_off(int row, int kr, int es) {
    const int kb = kr * es;
    return uint32_t((row >> 3) * (8 * TBKR * es) + (kb >> 4) * 128 + (row & 7) * 16 + (kb & 15));
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

// 3-D TMA tile load (shared::cluster destination = this CTA's own memory)
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// contiguous bulk copy global -> this CTA's shared memory (16-byte aligned,
// size a multiple of 16), completion counted on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Persistent warp-specialised kernel, five warpgroups.
//   warps 0-7  : B: streaming, per-thread cp.async pieces LOOK chunks ahead,
//                expanded chunk by chunk; resident / dictionary, the whole
//                B loaded and expanded at each group (column tile) switch.
//                BF16x3: A split into hi/lo from the TMA ring into TMEM; TF32
//                reads A straight from the ring.
//   warps 8-15 : epilogue, two warps per TMEM lane quadrant (warp % 4), each
//                draining 16 complex columns of each half tile; two
//                accumulators so that a tile's epilogue overlaps the next
//                tile's MMAs.
//   warp 16    : TMEM allocation; lane 0 issues tcgen05.mma and commits.
//   warp 17    : lane 0 streams A: one TMA tile load per chunk (128 rows x
//                16 complex k, 128-byte rows, swizzled) into a ring of RST
//                stages, several chunks ahead.
//   warp 18    : epilogue metadata (instances, rescale, C offsets, E_C),
//                a ring of MS tiles ahead of the epilogue.
// The epilogue warpgroups take registers from the others (setmaxnreg).
constexpr int NPROD = 256;   // warps 0-7
// BF16x3: warps 0-3 alone write the split A into TMEM, each thread one row
// (its warp's lane quadrant), both K steps.  With the two K steps written by
// warps w and w + 4 at once (same lanes, other columns) the products came
// out different from run to run; one writer per lane quadrant gives the
// exact results of the shared-memory form.
constexpr int NAW = 128;
constexpr int EPI_WARP0 = 8; // warps 8-15: two per TMEM lane quadrant
constexpr int NEPI = 256;
constexpr int MMA_WARP = 16;
constexpr int TMA_WARP = 17;
constexpr int META_WARP = 18;  // warp 19 idles
constexpr int NTHREADS = 640;
// Register split (setmaxnreg, per warpgroup).  The block is launched with
// 96 registers a thread (640 x 96 = 61440); after the split: producers
// 256 x 88 + epilogue 256 x 112 + control warpgroup 128 x 72 = 60416.
constexpr int LAUNCH_REGS = 96, PROD_REGS = 88, EPI_REGS = 112, CTL_REGS = 72;
static_assert(NPROD * PROD_REGS + NEPI * EPI_REGS + 128 * CTL_REGS <= NTHREADS * LAUNCH_REGS,
              "register split above the launch allocation");
constexpr int MS = 8;         // epilogue metadata ring (tiles ahead of the epilogue)
constexpr int NACC_MAX = 8;   // accumulators in TMEM (narrow tiles: up to 8 in flight)
constexpr int TMEM_COLS2 = 256;  // accumulators
// BF16x3 also keeps the split A chunks in TMEM, 32 columns a stage after
// the accumulators (at most 8 stages), so it allocates all 512 columns
constexpr int TM_A = TMEM_COLS2, TM_ASTAGE = 32;
// resident B: the TMEM A stages (8) run apart from the TMA ring (the ring
// slot is free once the producers have read it), so the A stream runs up
// to nrs + 8 chunks ahead of the MMAs; packed B ties a stage to its ring
// slot (the slot also holds the chunk's B)
constexpr int NTS = 8;
static_assert(TM_A + NTS * TM_ASTAGE <= 512, "TMEM A stages within the allocation");
template <int PREC>
__host__ __device__ constexpr uint32_t tmem_alloc_cols() { return PREC == 2 ? 512u : uint32_t(TMEM_COLS2); }

// Shared-memory layout.  Streaming B (BRES = false): A ring, B MMA stages,
// raw B pieces, epilogue staging.  Resident B (BRES = true): a pool of
// NSLOT 16 KB slots holding the A ring (first nrs slots) and the current
// group's whole B operand (the next nct x nch slots), then the staging.
template <int PREC, bool BRES>
struct Cfg {
    static constexpr int ST = PREC == 1 ? 4 : 3;      // MMA stages (streaming B)
    static constexpr int RST = BRES ? 8 : (PREC == 1 ? 4 : 6);  // A stages (most)
    static constexpr int BRST = 4;                    // raw B stages (per-thread cp.async pieces)
    static constexpr int LOOK = BRST - 1;             // B chunks issued ahead (streaming B)
    static constexpr int SLOT_RAW = TBM * TBK * 8;    // FP32 A chunk: 128 rows x 128 bytes, 128-byte swizzle
    static constexpr int SLOT_B = TBNR * TBKR * 4;    // one B chunk in MMA form (TF32, or BF16 hi + lo)
    static constexpr int SLOT_BRAW = TBN * TBK * 8;   // raw complex64 B chunk
    static constexpr int STAGE = 8 * 32 * 16 * 8;     // 4 KB per epilogue warp, in destination order
    static constexpr int NSLOT = 11;                  // resident-B pool
    static constexpr int OFF_RAW = 0;
    static constexpr int OFF_B = BRES ? 0 : OFF_RAW + RST * SLOT_RAW;
    static constexpr int OFF_BRAW = BRES ? 0 : OFF_B + ST * SLOT_B;
    static constexpr int OFF_STAGE = BRES ? NSLOT * SLOT_RAW : OFF_BRAW + BRST * SLOT_BRAW;
    static constexpr int OFF_CTRL = OFF_STAGE + STAGE;
    static_assert(SLOT_B == SLOT_RAW, "pool slots hold A or B chunks");
    static_assert(LOOK < BRST, "B pieces in flight fit the raw ring");
};
constexpr int BRES_MAX_B = 8;  // resident B: at most 8 chunks (nct x nch), so at least 3 A stages
constexpr int PACK_ST = 5;     // packed B: 5 stages of (A chunk, B chunk) in the pool
// packed B, column-tile pairs (MODE 4): 3 stages of (A chunk, B chunk of
// 256 real columns = 2 slots): slots 0-2 A, 3-8 B
constexpr int PAIR_ST = 3;
static_assert(2 * PACK_ST <= Cfg<2, true>::NSLOT && PACK_ST <= Cfg<2, true>::RST, "packed-B stages fit the pool");
static_assert(3 * PAIR_ST <= Cfg<2, true>::NSLOT, "paired packed-B stages fit the pool");

// Per-tile epilogue metadata, written by the metadata warp into a ring of
// MS slots ahead of the epilogue.
struct alignas(16) EpiMeta {
    int32_t inst[TBN];    // output instance of each column (-1: none)
    float sc[TBN];        // 2^-(ea + eb): the column's power-of-two rescale
    uint32_t mx[TBN];     // max-|component| of a run of an instance's columns, at the run's first column
    int16_t acol[TBN];    // B dictionary: accumulator (complex) column holding tile column c
    int64_t base;         // element offset of tile element (row 0, column 0) in C
    int32_t ncv, pad;     // valid columns
};

// Destination order of one epilogue warp's 32 rows x 16 complex columns.
// Its 9 tile bits (row bits 0-4 = lane, column bits 0-3) are sorted by the
// C offset they add; bit k of a compressed index is the k-th of them.
// Compressed neighbours land at neighbouring addresses wherever the C
// layout allows, so each store instruction covers one contiguous run.
struct EpiMap {
    int64_t doff[9];      // C offset of compressed bit k
    int64_t offI[8];      // C offset of compressed bits 6-8 = i (store round)
    int64_t qoff[4];      // C offset of row block 32q (row bits 5, 6)
    int64_t hoff[4];      // C offset of column block 16s (column bits 4, 5)
    int32_t colI[8];      // column of compressed bits 6-8 = i
    int32_t dcol[9];      // column of compressed bit k
    int32_t rank[9];      // compressed position of warp bit b (rows 0-4, columns 0-3)
    int32_t pair;         // doff[0] == 1: compressed elements 2u, 2u+1 are one 16-byte store
    int32_t nrows;        // valid rows per tile (min(M, 128))
    int32_t direct;       // narrow tiles with C bit 0 = row bit 0: each lane stores its row's columns
    int64_t coff[16];     // direct stores: C offset of tile column c (a group's columns start at 0)
};

struct Ctrl {
    uint64_t full[4], empty[4], rfull[8], rempty[8], afull[8], taempty[8], tfull[NACC_MAX], tempty[NACC_MAX],
        mfull[MS], mempty[MS];
    uint64_t bfull, bempty;  // resident B: loaded / no longer read by the MMAs
    uint32_t tmem_base;
    int32_t abort_;
    EpiMeta epi[MS];
    EpiMap map;
};

template <int PREC, bool BRES>
constexpr size_t smem_bytes() {
    return size_t(Cfg<PREC, BRES>::OFF_CTRL) + sizeof(Ctrl) + 1024;
}
static_assert(smem_bytes<1, false>() <= 232448 && smem_bytes<2, false>() <= 232448 &&
                  smem_bytes<1, true>() <= 232448 && smem_bytes<2, true>() <= 232448,
              "shared memory above 227 KB");

// Tile T of a step.  Schedule 0: the tiles of one group (its column tiles
// x row tiles) are numbered row tile major, column tile minor, so the
// column tiles that share an A row tile run on neighbouring CTAs and A is
// read from DRAM about once.  Schedule 1: column tile major, row tile minor
// (the B columns of a column tile stay in L2 across its row tiles).  Returns the column-tile record with its first column, and
// the row tile in mt.
__device__ __forceinline__ int4 tile_decode(const StepDesc &d, int64_t T, int64_t mtiles, int64_t &mt,
                                            int64_t *group = nullptr) {
    const int64_t e0 = T / mtiles;  // some column tile of T's group
    int4 r = __ldg(d.trec + e0);
    const int64_t f = e0 - r.w / TBN;  // the group's first column tile
    // resident-B unit: the group (schedule 0) or the column tile (schedule 1)
    if (group) *group = d.sched != 0 ? e0 : f;
    if (d.sched != 0) {  // schedule 1: the row tiles of one column tile run consecutively
        mt = T - e0 * mtiles;
        return r;
    }
    const int64_t nct = ((int64_t(r.y) << d.nb) + TBN - 1) / TBN;
    const int64_t local = T - f * mtiles;
    mt = local / nct;
    r.w = int((local - mt * nct) * TBN);
    return r;
}

// Walks a CTA's contiguous range of tiles in order.  One division at the
// start (tile_decode's); afterwards each step is a counter update, and the
// column-tile record of the next unit (schedule 1: the next column tile;
// schedule 0: the next group) is fetched one unit ahead, so no role waits on
// a global load per tile.
struct TileIter {
    int64_t f;       // unit: schedule 1 its column-tile record, schedule 0 its group's first record
    int mt;          // row tile
    int ct, nct;     // column tile within the unit and their count (schedule 1: 0 and 1)
    int4 rec, nrec;  // the unit's record (schedule 0: its first, column offset 0) and the next unit's
    // blocks of tblk tiles dealt round-robin to the CTAs (tblk = 0: one
    // contiguous range per CTA): the next block's first tile, the tiles
    // left in the current block
    int64_t bnext;
    int bleft;
    // pp: column-tile pairs of N = 64 steps, each group's column tiles
    // padded to an even count nctp (the pad tile has no valid columns);
    // tile indices count padded tiles (d.ptab)
    bool pp;
    int nctp;

    __device__ __forceinline__ static int unit_tiles(const StepDesc &d, const int4 &r) {
        return d.sched != 0 ? 1 : int(((int64_t(r.y) << d.nb) + TBN - 1) / TBN);
    }
    __device__ __forceinline__ void fetch_next(const StepDesc &d) {
        const int64_t fn = f + nct;
        nrec = fn < d.n_ctab ? __ldg(d.trec + fn) : make_int4(0, 0, 0, 0);
    }
    __device__ __forceinline__ void init(const StepDesc &d, int64_t T, int64_t mtiles) {
        if (pp) {
            const int2 q = __ldg(d.ptab + T / mtiles);  // {group's first column tile, its first padded one}
            f = q.x;
            rec = __ldg(d.trec + f);  // column offset 0
            nct = unit_tiles(d, rec);
            nctp = nct + (nct & 1);
            const int64_t local = T - int64_t(q.y) * mtiles;
            mt = int(local / nctp);
            ct = int(local - int64_t(mt) * nctp);
            fetch_next(d);
            return;
        }
        int64_t m, g;
        rec = tile_decode(d, T, mtiles, m, &g);
        f = g;
        mt = int(m);
        ct = 0;
        if (d.sched == 0) {
            ct = rec.w / TBN;
            rec.w = 0;
        }
        nct = unit_tiles(d, rec);
        nctp = nct;
        fetch_next(d);
    }
    // the current tile's record (first instance, count, A instance, first column)
    __device__ __forceinline__ int4 record(const StepDesc &d) const {
        int4 r = rec;
        if (d.sched == 0) r.w = ct * TBN;
        return r;
    }
    // the CTA's first tile (blocks: its first block's)
    __device__ __forceinline__ void start(const StepDesc &d, int64_t mtiles, int64_t n_tiles, int tblk,
                                          bool padded = false) {
        pp = padded;
        if (tblk <= 0) {
            bleft = 0x7fffffff;
            init(d, n_tiles * blockIdx.x / gridDim.x, mtiles);
            return;
        }
        const int64_t t0 = int64_t(blockIdx.x) * tblk;
        bleft = int(min(int64_t(tblk), n_tiles - t0));
        bnext = t0 + int64_t(gridDim.x) * tblk;
        init(d, t0, mtiles);
    }
    __device__ __forceinline__ void next(const StepDesc &d, int64_t mtiles, int64_t n_tiles, int tblk) {
        if (tblk > 0 && --bleft == 0) {  // the CTA's next block
            if (bnext < n_tiles) {
                bleft = int(min(int64_t(tblk), n_tiles - bnext));
                init(d, bnext, mtiles);
                bnext += int64_t(gridDim.x) * tblk;
            }
            return;
        }
        if (++ct < nctp) return;
        ct = 0;
        if (++mt < mtiles) return;
        mt = 0;
        f += nct;
        rec = nrec;
        nct = unit_tiles(d, rec);
        nctp = pp ? nct + (nct & 1) : nct;
        fetch_next(d);
    }
};

// XOR swizzle of a warp staging area (256 16-byte units): eight consecutive
// units stay within one 128-byte row, and units that differ in higher bits
// spread over the banks
__device__ __forceinline__ int stage_swz(int u) { return u ^ (((u >> 3) ^ (u >> 6)) & 7); }

// One producer thread's B piece: column bcol, complex k 4 kqb .. 4 kqb + 3
// of a chunk (p0, p1 = the four values), expanded into the real 2x2 form
// (rows 2 bcol: Re, -Im; 2 bcol + 1: Im, Re) in the K-major no-swizzle
// layout of a B chunk of nr rows (MMA N: 128, or 256 for a column-tile
// pair); BF16x3 stores the hi plane, then the lo plane nr x 64 bytes on.
template <int PREC, bool RM = false>
__device__ __forceinline__ void expand_b(uint8_t *base, int bcol, int kqb, const float4 p0, const float4 p1,
                                         int nr = TBNR) {
    // RM: row-group-major order (rmaj_off; nr = TBNR)
    auto off = [&](int row, int kr, int es) { return RM ? rmaj_off(row, kr, es) : kmaj_off(row, kr, es, nr); };
    const float2 t4[4] = {make_float2(p0.x, p0.y), make_float2(p0.z, p0.w), make_float2(p1.x, p1.y),
                          make_float2(p1.z, p1.w)};
    const float r0[8] = {t4[0].x, -t4[0].y, t4[1].x, -t4[1].y, t4[2].x, -t4[2].y, t4[3].x, -t4[3].y};
    const float r1[8] = {t4[0].y, t4[0].x, t4[1].y, t4[1].x, t4[2].y, t4[2].x, t4[3].y, t4[3].x};
    // A 16-byte unit's bank group is its row mod 8, so the threads of a
    // warp (32 consecutive columns) write the odd row first where bit 2 of
    // the column is set: each store instruction then covers all 32 banks
    const int sw = (bcol >> 2) & 1;
    const int ra = 2 * bcol + sw, rb = 2 * bcol + 1 - sw;
    if (PREC == 1) {
        const float4 a0 = make_float4(r0[0], r0[1], r0[2], r0[3]), a1 = make_float4(r0[4], r0[5], r0[6], r0[7]);
        const float4 b0 = make_float4(r1[0], r1[1], r1[2], r1[3]), b1 = make_float4(r1[4], r1[5], r1[6], r1[7]);
        *reinterpret_cast<float4 *>(base + off(ra, 8 * kqb, 4)) = sw ? b0 : a0;
        *reinterpret_cast<float4 *>(base + off(ra, 8 * kqb + 4, 4)) = sw ? b1 : a1;
        *reinterpret_cast<float4 *>(base + off(rb, 8 * kqb, 4)) = sw ? a0 : b0;
        *reinterpret_cast<float4 *>(base + off(rb, 8 * kqb + 4, 4)) = sw ? a1 : b1;
    } else {
        __align__(16) __nv_bfloat16 h0[8], l0[8], h1[8], l1[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            h0[q] = __float2bfloat16_rn(r0[q]);
            l0[q] = __float2bfloat16_rn(r0[q] - __bfloat162float(h0[q]));
            h1[q] = __float2bfloat16_rn(r1[q]);
            l1[q] = __float2bfloat16_rn(r1[q] - __bfloat162float(h1[q]));
        }
        uint8_t *blo = base + nr * TBKR * 2;
        const uint4 H0 = *reinterpret_cast<uint4 *>(h0), L0 = *reinterpret_cast<uint4 *>(l0);
        const uint4 H1 = *reinterpret_cast<uint4 *>(h1), L1 = *reinterpret_cast<uint4 *>(l1);
        const uint32_t oa = off(ra, 8 * kqb, 2), ob = off(rb, 8 * kqb, 2);
        *reinterpret_cast<uint4 *>(base + oa) = sw ? H1 : H0;
        *reinterpret_cast<uint4 *>(blo + oa) = sw ? L1 : L0;
        *reinterpret_cast<uint4 *>(base + ob) = sw ? H0 : H1;
        *reinterpret_cast<uint4 *>(blo + ob) = sw ? L0 : L1;
    }
}

// BF16x3: the A operand goes to tensor memory.  A chunk arrives by TMA as
// 128 rows of 32 real k (128 bytes, 128-byte swizzle).  The A stage in TMEM
// is 32 columns (128 lanes = rows): K step h (16 real k, 8 columns of
// packed bf16 pairs, lower k in the low half) holds hi in columns
// 16 h .. 16 h + 7 and lo in the next 8.  The MMAs then read only B from
// shared memory.
//
// Quarter q (real k 8 q .. 8 q + 7, logical 16-byte units 2 q, 2 q + 1) of
// this thread's row: read from the swizzled slot, split into hi and lo,
// stored to hi columns 16 (q / 2) + 4 (q % 2) .. + 3 and the lo columns 8
// further on, relative to ta (this lane's row of the stage).  tcgen05.st is
// warp-wide (.sync.aligned).
__device__ __forceinline__ void split_a_quarter(const uint8_t *slot, int row, int q, uint32_t ta) {
    const int sw = row & 7;
    const uint8_t *rowp = slot + row * 128;
    const float4 v0 = *reinterpret_cast<const float4 *>(rowp + (((2 * q) ^ sw) << 4));
    const float4 v1 = *reinterpret_cast<const float4 *>(rowp + (((2 * q + 1) ^ sw) << 4));
    const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * p], x[2 * p + 1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(x[2 * p] - hf.x, x[2 * p + 1] - hf.y);
        hw[p] = *reinterpret_cast<const uint32_t *>(&h);
        lw[p] = *reinterpret_cast<const uint32_t *>(&lo);
    }
    const uint32_t c = ta + uint32_t(16 * (q >> 1) + 4 * (q & 1));
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(c), "r"(hw[0]), "r"(hw[1]),
                 "r"(hw[2]), "r"(hw[3])
                 : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(c + 8u), "r"(lw[0]), "r"(lw[1]),
                 "r"(lw[2]), "r"(lw[3])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Resident B: the producer threads load the B operand of a group's column
// tiles ct0 .. ct0 + nct - 1 (schedule 0: all of the group's; schedule 1:
// the tile's own; dictionary: every B instance of the step, instance j in
// columns jN .. jN + N - 1), nch K chunks each, zeros past its columns and past K,
// into pool slots bset[(ct - ct0) * nch + c], two chunks' global loads in
// flight per thread at a time.  Each column is multiplied by its power-of-two
// rescale 2^-(ea + eb) on the way (exact), so the epilogue stores the
// accumulators as they are.
template <int PREC, bool DICT>
__device__ __forceinline__ void load_bset(const StepDesc &d, const int4 &r, int nch, int K, uint8_t *bset,
                                          int bcol, int kqb) {
    const int64_t ncols = DICT ? (d.nInstB << d.nb) : int64_t(r.y) << d.nb;
    const int ct0 = (!DICT && d.sched != 0) ? r.w / TBN : 0;
    const int nct = (DICT || d.sched != 0) ? 1 : int((ncols + TBN - 1) / TBN);
    const int N = 1 << d.nb;
    // dictionary: column gc is column gc mod N of B instance gc / N, scaled
    // by 2^-eb only (the A exponent changes from group to group)
    const int ea = (!DICT && d.mxA) ? exp_of(__ldg(d.mxA + r.z)) : 0;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int ct = 0; ct < nct && ct < BRES_MAX_B; ++ct) {
        // this thread's column in the column tile: element offset in B (or
        // -1) and its power-of-two rescale 2^-(ea + eb), applied here
        // instead of in the epilogue
        const int64_t gc = int64_t(ct0 + ct) * TBN + bcol;
        int64_t bb = -1;
        float s = 1.f;
        if (gc < ncols) {
            const int ib = DICT ? int(gc >> d.nb) : __ldg(d.instab + r.x + (gc >> d.nb)).y;
            bb = int64_t(ib) * d.sB + ((gc & (N - 1)) << d.kb);
            s = pow2f(-(ea + (d.mxB ? exp_of(__ldg(d.mxB + ib)) : 0)));
        }
        for (int c = 0; c < nch; c += 2) {
            float4 p[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int k = (c + i) * TBK + 4 * kqb;
                const bool v = bb >= 0 && c + i < nch && k + 3 < K;
                const float4 *src = reinterpret_cast<const float4 *>(v ? d.B + bb + k : d.B);
                p[i][0] = v ? __ldg(src) : z;
                p[i][1] = v ? __ldg(src + 1) : z;
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
                if (c + i < nch)
                    expand_b<PREC>(bset + (ct * nch + c + i) * (TBNR * TBKR * 4), bcol, kqb,
                                   make_float4(p[i][0].x * s, p[i][0].y * s, p[i][0].z * s, p[i][0].w * s),
                                   make_float4(p[i][1].x * s, p[i][1].y * s, p[i][1].z * s, p[i][1].w * s));
        }
    }
}

// tcgen05.ld of NR consecutive 32-bit accumulator columns (32x32b shape:
// lane i of the warp gets row i of its lane quadrant)
template <int NR>
__device__ __forceinline__ void tmem_ld(uint32_t ta, uint32_t *r) {
    if constexpr (NR == 2) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(ta));
    } else if constexpr (NR == 4) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                     : "r"(ta));
    } else if constexpr (NR == 8) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(ta));
    } else if constexpr (NR == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(ta));
    } else {
        static_assert(NR == 16, "32 columns at most");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta));
    }
}

// B dictionary, a warp block of 16 columns c0 .. c0 + 15: every run of R
// columns (one instance) from the accumulator columns its instance's B
// occupies; all loads issued before one wait.  Columns past the tile's
// valid ones read as zeros.
template <int NC, int R>
__device__ __forceinline__ void tmem_gather16(uint32_t (&r)[32], uint32_t tb, const EpiMeta &em, int c0, int ncv) {
#pragma unroll
    for (int j = 0; j < NC / R; ++j) tmem_ld<2 * R>(tb + 2u * uint32_t(em.acol[c0 + j * R]), r + 2 * j * R);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < NC / R; ++j) {
        const bool ok = c0 + j * R < ncv;
#pragma unroll
        for (int q = 0; q < 2 * R; ++q) r[2 * j * R + q] = ok ? r[2 * j * R + q] : 0u;
    }
}

// Max-|component| of a warp block (16 complex columns; r: this lane's 32
// accumulator values as float bits) over runs of RUN columns (one instance
// each): folded in registers, one warp reduction per run, scaled by the
// run's power of two (exact; SCALED: the values carry it already) and merged
// into the slot's entry at the run's first column.  Columns past the tile's
// valid ones hold zeros and merge nothing.
template <int NC, int RUN, bool SCALED>
__device__ __forceinline__ void fold_max16(const uint32_t (&r)[32], EpiMeta &em, int c0, int lane) {
    uint32_t a[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j)
        a[j] = __float_as_uint(fmaxf(fabsf(__uint_as_float(r[2 * j])), fabsf(__uint_as_float(r[2 * j + 1]))));
#pragma unroll
    for (int s = 1; s < RUN; s <<= 1)
#pragma unroll
        for (int j = 0; j < NC; j += 2 * s) a[j] = max(a[j], a[j + s]);
#pragma unroll
    for (int j = 0; j < NC; j += RUN) {
        const uint32_t m = __reduce_max_sync(0xffffffffu, a[j]);
        if (lane == 0 && m)
            atomicMax(&em.mx[c0 + j], SCALED ? m : __float_as_uint(__uint_as_float(m) * em.sc[c0 + j]));
    }
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)  // 20 warps: 96 registers (5 warps on a sub-partition)
    k_step_gemm_tc(const __grid_constant__ StepDesc d, int64_t mtiles, int32_t *err, const __grid_constant__ CUtensorMap tmA, int nrs,
                   int acw, int ow, int tblk) {
    // MODE 0: B streamed chunk by chunk; 1: B resident (a group's or a
    // column tile's), rescale folded into it; 2: B dictionary, every B
    // instance of the step (at most 64 columns) resident for the whole
    // launch, each tile's columns gathered from the accumulator.
    // nrs: A stages in use (C::RST streaming B; resident B: the pool slots
    // left after the largest resident B)
    // acw: complex columns of an accumulator (8, 16, 32 or 64; MMA N =
    // 2 acw): the widest tile (MODE 0, 1) or the dictionary (MODE 2), so
    // that narrow steps do not multiply zero columns; 128 / acw accumulators
    // (at most NACC_MAX) rotate through TMEM.  ow: most output columns of a
    // tile (8 .. 64).  With ow <= 16 the two halves of the epilogue (warps
    // 8-11, 12-15) drain alternate tiles, each warp 32 rows x ow columns.
    // MODE 3: B packed in MMA form in global memory (tc_pack_b, once per
    // launch) and bulk-copied chunk by chunk beside A from L2, B carrying
    // 2^-eb
    constexpr bool BRES = MODE == 1 || MODE == 2;
    // MODE 4: packed B with two adjacent column tiles of a row tile (one B
    // instance's 128 columns, or with N = 64 two instances' 64) per MMA of
    // N = 256, both accumulators at once
    constexpr bool PAIR = MODE == 4;
    constexpr bool BPACK = MODE == 3 || PAIR;
    constexpr int TSTEP = PAIR ? 2 : 1;  // tiles per unit of A / MMA work
    // pairs with N = 64: the pair's two column tiles are two instances of
    // the group (B packed per instance in row-group-major order, four bulk
    // copies per chunk), groups padded to an even tile count
    const bool PP = PAIR && d.nb == 6;
    using C = Cfg<PREC, BRES || BPACK>;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment: the swizzled A slots are whole 8-row atoms
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Ctrl &X = *reinterpret_cast<Ctrl *>(sm + C::OFF_CTRL);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = (PP ? d.n_ptab : d.n_ctab) * mtiles;
    const int N = 1 << d.nb;
    const int K = 1 << d.kb;
    const int nch = (K + TBK - 1) / TBK;
    // accumulators in rotation: a power of two, so tile l uses accumulator
    // l & (nacc - 1) in its phase l >> nacc_sh (no 64-bit division)
    const int nacc_sh = acw >= 64 ? 1 : (acw == 32 ? 2 : 3);
    const int nacc = 1 << nacc_sh;
    static_assert(NACC_MAX == 8, "accumulator rotation of at most 8");
    const uint32_t awr = uint32_t(2 * acw);  // TMEM columns of an accumulator
    const bool narrow = ow <= 16;
    const int nepi = narrow ? NEPI / 2 : NEPI;  // epilogue threads that drain one tile
    // one contiguous range of tiles per CTA (a unit's tiles run back to
    // back: its B and its records are reused)
    // tblk = 0: one contiguous range of tiles per CTA; else blocks of tblk
    // tiles dealt round-robin, so that the CTAs work on neighbouring tiles
    // at any time (their A and B stay in L2)
    int64_t my_tiles;
    if (tblk <= 0) {
        my_tiles = n_tiles * (blockIdx.x + 1) / gridDim.x - n_tiles * blockIdx.x / gridDim.x;
    } else {
        const int64_t nblk = (n_tiles + tblk - 1) / tblk;
        const int64_t mine = nblk > blockIdx.x ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        my_tiles = mine * tblk;
        if (mine > 0 && (blockIdx.x + (mine - 1) * int64_t(gridDim.x)) == nblk - 1) my_tiles -= nblk * tblk - n_tiles;
    }
    const int64_t total_chunks = my_tiles * nch;

    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&X.tmem_base)),
                     "r"(tmem_alloc_cols<PREC>())
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
            // BF16x3 (not packed B): the producers release the A slot once
            // they hold its values; otherwise the MMAs' commit does
            mbar_init(&X.rempty[s], (PREC == 2 && !BPACK) ? NAW : 1);
        }
        for (int s = 0; s < NTS; ++s) {
            mbar_init(&X.afull[s], NAW);
            mbar_init(&X.taempty[s], 1);
        }
        mbar_init(&X.bfull, PREC == 1 ? NPROD : NPROD - NAW);  // the resident-B loaders
        mbar_init(&X.bempty, 1);
        for (int a = 0; a < NACC_MAX; ++a) {
            mbar_init(&X.tfull[a], 1);
            mbar_init(&X.tempty[a], nepi);
        }
        for (int s = 0; s < MS; ++s) {
            mbar_init(&X.mfull[s], 32);
            mbar_init(&X.mempty[s], nepi);
        }
        X.abort_ = *reinterpret_cast<volatile int32_t *>(err);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // destination order of an epilogue warp's block (same for every tile)
        EpiMap &mp = X.map;
        constexpr int64_t NONE = 0x7fffffffffffffffLL;  // row bits at or above mb: never stored
        auto rowkey = [&](int b) -> int64_t { return b < d.mb ? (int64_t(1) << d.pCm[b]) : NONE; };
        auto colkey = [&](int j) -> int64_t { return j < d.nb ? (int64_t(1) << d.pCn[j]) : (d.sC << (j - d.nb)); };
        // rank of each bit by destination stride (ties by index); unrolled
        // so that the keys stay in registers
        int64_t key[9];
#pragma unroll
        for (int b = 0; b < 5; ++b) key[b] = rowkey(b);
#pragma unroll
        for (int j = 0; j < 4; ++j) key[5 + j] = colkey(j);
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            int k = 0;
#pragma unroll
            for (int a = 0; a < 9; ++a) k += (key[a] < key[b] || (key[a] == key[b] && a < b)) ? 1 : 0;
            mp.rank[b] = k;
            mp.doff[k] = key[b];
            mp.dcol[k] = b < 5 ? 0 : (1 << (b - 5));
        }
        for (int i = 0; i < 8; ++i) {
            int64_t o = 0;
            int c = 0;
            for (int k = 6; k < 9; ++k)
                if ((i >> (k - 6)) & 1) {
                    o += mp.doff[k];
                    c += mp.dcol[k];
                }
            mp.offI[i] = o;
            mp.colI[i] = c;
        }
        for (int q = 0; q < 4; ++q) {
            mp.qoff[q] = ((q & 1) && d.mb > 5 ? rowkey(5) : 0) + ((q & 2) && d.mb > 6 ? rowkey(6) : 0);
            mp.hoff[q] = ((q & 1) ? colkey(4) : 0) + ((q & 2) ? colkey(5) : 0);
        }
        mp.pair = mp.doff[0] == 1;
        mp.nrows = d.mb >= 7 ? TBM : (1 << d.mb);
        // Narrow tiles (one tile per group, at most 8 columns) whose C
        // layout puts row bit 0 at address bit 0: lanes (rows) store
        // neighbouring elements, so the registers go out without staging
        mp.direct = (ow <= 8 && d.mb >= 7 && d.pCm[0] == 0) ? 1 : 0;
        for (int c = 0; c < 16; ++c)
            mp.coff[c] = c < (1 << d.nb) * d.max_group
                             ? int64_t(c >> d.nb) * d.sC + dep(int64_t(c & ((1 << d.nb) - 1)), d.pCn, d.nb)
                             : 0;
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

    if (warp >= MMA_WARP) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(CTL_REGS));
    if (warp == TMA_WARP) {
        // ------------------------------------------------------------ A stream
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            int64_t issued = 0;
            bool ok = true;
            TileIter it;
            if (my_tiles > 0) it.start(d, mtiles, n_tiles, tblk, PP);
            int rs = 0;
            uint32_t rph = 0;
            const uint8_t *bsrc = nullptr;   // packed B: the tile's first chunk
            const uint8_t *bsrc1 = nullptr;  // N = 64 pairs: the second tile's
            int64_t fprev = -1;
            int ctprev = -1;
            for (int64_t l = 0; l < my_tiles && ok && !*abort_flag; l += TSTEP) {
                const int4 r = it.record(d);
                const int m0 = int(it.mt * TBM);
                if (BPACK && (it.f != fprev || it.ct != ctprev)) {
                    const int64_t i0 = int64_t(r.x) + (r.w >> d.nb);
                    const int ib = __ldg(d.instab + i0).y;
                    if (PP) {
                        // N = 64: tile ct is instance ct of the group; the
                        // pad tile (odd groups) repeats the first tile's B
                        const int ib1 = it.ct + 1 < it.nct ? __ldg(d.instab + i0 + 1).y : ib;
                        bsrc = d.bpack + int64_t(ib) * nch * C::SLOT_B;
                        bsrc1 = d.bpack + int64_t(ib1) * nch * C::SLOT_B;
                    } else {
                        // the tile's 64 columns (a pair's 128) lie in one B
                        // instance (N >= 64, pairs N >= 128): its chunks for
                        // this column tile (pair) are consecutive
                        const int pb = PAIR ? 7 : 6;
                        const int64_t blk = (int64_t(ib) << (d.nb - pb)) + ((r.w & (N - 1)) >> pb);
                        bsrc = d.bpack + blk * nch * int64_t(TSTEP * C::SLOT_B);
                    }
                    fprev = it.f;
                    ctprev = it.ct;
                }
                for (int c = 0; c < nch; ++c, ++issued) {
                    if (!mbar_wait(&X.rempty[rs], rph ^ 1u)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&X.rfull[rs], BPACK ? C::SLOT_RAW + TSTEP * C::SLOT_B : C::SLOT_RAW);
                    tma_load_3d(smem_u32(sm + C::OFF_RAW + rs * C::SLOT_RAW), &tmA, TBKR * c, m0, r.z, &X.rfull[rs]);
                    const uint32_t bdst = smem_u32(sm + C::OFF_RAW + (PAIR ? PAIR_ST + 2 * rs : PACK_ST + rs) * C::SLOT_RAW);
                    if (PP) {  // hi planes of both tiles, then both lo planes
                        constexpr int PL = C::SLOT_B / 2;
                        const uint8_t *s0 = bsrc + int64_t(c) * C::SLOT_B, *s1 = bsrc1 + int64_t(c) * C::SLOT_B;
                        bulk_load(bdst, s0, PL, &X.rfull[rs]);
                        bulk_load(bdst + PL, s1, PL, &X.rfull[rs]);
                        bulk_load(bdst + 2 * PL, s0 + PL, PL, &X.rfull[rs]);
                        bulk_load(bdst + 3 * PL, s1 + PL, PL, &X.rfull[rs]);
                    } else if (BPACK) {
                        bulk_load(bdst, bsrc + c * TSTEP * C::SLOT_B, TSTEP * C::SLOT_B, &X.rfull[rs]);
                    }
                    if (++rs == nrs) {
                        rs = 0;
                        rph ^= 1u;
                    }
                }
                for (int t = 0; t < TSTEP; ++t) it.next(d, mtiles, n_tiles, tblk);
            }
            if (!ok) give_up();
            // loads still in flight land before the CTA leaves (bounded)
            for (int64_t j = issued > nrs ? issued - nrs : 0; j < issued; ++j)
                mbar_wait(&X.rfull[j % nrs], uint32_t(j / nrs) & 1u);
        }
        __syncwarp();
    } else if (warp < NPROD / 32) {
        // ------------------------------------------------------------ B loads, A split
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(PROD_REGS));
        const int bcol = tid & 63, kqb = tid >> 6;
        // BF16x3 A (warps 0-3): this thread's row, its warp's TMEM lane
        // quadrant
        const bool awriter = PREC == 2 && warp < NAW / 32;
        const int arow = 32 * (warp & 3) + lane;
        const uint32_t ta_row = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(TM_A);
        // one chunk of A from the TMA slot into TMEM stage `stage` (both K
        // steps); the slot is released once read (rel: its barrier, or null)
        auto a_to_tmem = [&](const uint8_t *slot, int stage, uint64_t *rel) {
            const uint32_t ta = ta_row + uint32_t(stage * TM_ASTAGE);
            split_a_quarter(slot, arow, 0, ta);
            split_a_quarter(slot, arow, 1, ta);
            split_a_quarter(slot, arow, 2, ta);
            split_a_quarter(slot, arow, 3, ta);
            if (rel) mbar_arrive(rel);
        };
        // loop exits and waits are made warp-uniform: the TMEM stores below
        // are warp-wide instructions
        auto aborted = [&]() { return __any_sync(0xffffffffu, *abort_flag != 0); };
      if constexpr (BRES || BPACK) {
        // resident B: at each group switch (once the MMAs stopped reading
        // the previous group's B) the group's B goes into the pool -- BF16x3:
        // by warps 4-7 (two k quads per thread), while warps 0-3 split every
        // A chunk into a TMEM stage, so that neither loop carries the other's
        // registers; TF32: by all producer warps
        if (BRES && (PREC == 1 || warp >= NAW / 32)) {
            uint32_t u = 0;
            int64_t gprev = -1;
            TileIter it;
            if (my_tiles > 0) it.start(d, mtiles, n_tiles, tblk, PP);
            for (int64_t l = 0; l < my_tiles && !aborted(); ++l) {
                const int4 r = it.record(d);
                const int64_t g = MODE == 2 ? 0 : it.f;  // the dictionary is loaded once
                it.next(d, mtiles, n_tiles, tblk);
                if (g == gprev) continue;
                if (u > 0 && !__all_sync(0xffffffffu, mbar_wait(&X.bempty, (u - 1) & 1u))) {
                    give_up();
                    break;
                }
                uint8_t *bset = sm + C::OFF_RAW + nrs * C::SLOT_RAW;
                if constexpr (BRES) {
                    if (PREC == 1) {
                        load_bset<PREC, MODE == 2>(d, r, nch, K, bset, bcol, kqb);
                    } else {
#pragma unroll 1
                        for (int q = (tid - NAW) >> 6; q < 4; q += 2)  // k quads 0, 2 or 1, 3
                            load_bset<PREC, MODE == 2>(d, r, nch, K, bset, bcol, q);
                    }
                }
                proxy_fence();
                mbar_arrive(&X.bfull);
                ++u;
                gprev = g;
                if (MODE == 2) break;  // the dictionary: one load for the launch
            }
        } else if (awriter) {
            int rs = 0, ts = 0;
            uint32_t rph = 0, tph = 0;
            const int nts = BPACK ? nrs : NTS;
            bool ok = true;
            for (int64_t l = 0; l < my_tiles && ok && !aborted(); l += TSTEP) {
                for (int c = 0; c < nch; ++c) {
                    // the chunk has landed and the MMAs are done with the
                    // TMEM stage's previous chunk
                    bool w = mbar_wait(&X.rfull[rs], rph);
                    w = w && mbar_wait(&X.taempty[ts], tph ^ 1u);
                    if (!__all_sync(0xffffffffu, w)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // packed B: the slot pair waits for the MMAs
                    a_to_tmem(sm + C::OFF_RAW + rs * C::SLOT_RAW, ts, !BPACK ? &X.rempty[rs] : nullptr);
                    tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&X.afull[ts]);
                    if (++rs == nrs) {
                        rs = 0;
                        rph ^= 1u;
                    }
                    if (++ts == nts) {
                        ts = 0;
                        tph ^= 1u;
                    }
                }
            }
            if (!ok) give_up();
        }
      } else {
        int64_t issued = 0;
        // the B column of this thread, per unit and column tile: its
        // element offset in B (-1: past the tile's columns), looked up when
        // the tile's record or column offset changes
        int64_t bb = -1, fprev = -1;
        int ctprev = -1;
        int c_iss = 0;  // chunk of the tile being issued
        TileIter it;
        if (my_tiles > 0) it.start(d, mtiles, n_tiles, tblk, PP);
        for (int64_t gch = 0; gch < total_chunks && !aborted(); ++gch) {
            // B pieces run LOOK chunks ahead.  Each thread reads back only
            // the 32 bytes it copied, and its raw slot was last used by a
            // chunk it has already expanded, so the ring needs no barrier.
            while (issued < total_chunks && issued <= gch + C::LOOK) {
                const int c = c_iss;
                const int bslot = int(issued % C::BRST);
                if (c == 0) {
                    if (issued > 0) it.next(d, mtiles, n_tiles, tblk);
                    if (it.f != fprev || it.ct != ctprev) {
                        const int4 r = it.record(d);
                        const int64_t gc = int64_t(r.w) + bcol;
                        // column-affine B: column n of instance ib starts at ib*sB + n*K
                        bb = -1;
                        if (gc < (int64_t(r.y) << d.nb)) {
                            const int ib = __ldg(d.instab + (int64_t(r.x) + (gc >> d.nb))).y;
                            bb = int64_t(ib) * d.sB + ((gc & (N - 1)) << d.kb);
                        }
                        fprev = it.f;
                        ctprev = it.ct;
                    }
                }
                if (++c_iss == nch) c_iss = 0;
                {  // B: this thread's column, k quad kqb (its two 16-byte
                   // halves in the order that spreads a warp over all banks)
                    const uint32_t dst = smem_u32(sm + C::OFF_BRAW + bslot * C::SLOT_BRAW) + uint32_t(tid) * 32;
                    const int k = c * TBK + 4 * kqb;
                    const bool v = bb >= 0 && k + 3 < K;
                    const float2 *src = v ? d.B + bb + k : d.B;
                    const int h = (tid >> 2) & 1;
                    cp_async16(dst + 16 * h, v ? src + 2 * h : d.B, v ? 16 : 0);
                    cp_async16(dst + 16 * (1 - h), v ? src + 2 * (1 - h) : d.B, v ? 16 : 0);
                }
                cp_async_commit();
                ++issued;
            }
            const int slot = int(gch % C::ST);
            // the MMA stage (B slot, BF16x3: and the TMEM A stage of the
            // same index) is free once the MMAs of chunk gch - ST are done
            const int rs = int(gch % C::RST);
            bool w = mbar_wait(&X.empty[slot], (uint32_t(gch / C::ST) & 1u) ^ 1u);
            if (awriter) w = w && mbar_wait(&X.rfull[rs], uint32_t(gch / C::RST) & 1u);
            if (!__all_sync(0xffffffffu, w)) {
                give_up();
                break;
            }
            if (awriter) {  // A: into the TMEM stage; the TMA slot is free once read
                tc_fence_after();
                a_to_tmem(sm + C::OFF_RAW + rs * C::SLOT_RAW, slot, &X.rempty[rs]);
            }
            cp_async_wait(int(issued - gch - 1));
            // B: expand this thread's prefetched piece into the MMA layout
            {
                const uint8_t *braw = sm + C::OFF_BRAW + int(gch % C::BRST) * C::SLOT_BRAW + tid * 32;
                const int h = (tid >> 2) & 1;
                const float4 q0 = *reinterpret_cast<const float4 *>(braw + 16 * h);
                const float4 q1 = *reinterpret_cast<const float4 *>(braw + 16 * (1 - h));
                expand_b<PREC>(sm + C::OFF_B + slot * C::SLOT_B, bcol, kqb, h ? q1 : q0, h ? q0 : q1);
            }
            if (awriter) tmem_wait_st();
            proxy_fence();
            if (PREC == 2) tc_fence_before();
            mbar_arrive(&X.full[slot]);
        }
        cp_async_wait(0);
      }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t LBO = TBM * 16, SBO = 128;
            // the MMAs of one K chunk: A slot a0 (swizzled rows), B slot b0
            auto issue_chunk = [&](uint32_t dtm, uint32_t a0, uint32_t b0, bool first) {
                if (PREC == 1) {
                    const uint32_t id = idesc(2u, awr);
#pragma unroll
                    for (int j = 0; j < TBKR / 8; ++j) {  // K step: 8 tf32 = 32 bytes of an A row
                        const uint32_t off = uint32_t(2 * j) * LBO;
                        mma_tf32(dtm, sdesc_sw128(a0 + 32 * j), sdesc(b0 + off, LBO, SBO), id, (!first || j > 0) ? 1u : 0u);
                    }
                } else {
                    // A: the TMEM stage at column a0 (K step j: hi at
                    // a0 + 16 j, lo 8 columns on); B: hi plane, lo plane
                    // 8 KB on
                    const uint32_t id = idesc(1u, awr);
                    const uint32_t bl = b0 + TBNR * TBKR * 2;
#pragma unroll
                    for (int j = 0; j < TBKR / 16; ++j) {
                        const uint32_t off = uint32_t(2 * j) * LBO;
                        const uint32_t ah = a0 + uint32_t(16 * j), al = ah + 8u;
                        mma_f16_ts(dtm, ah, sdesc(b0 + off, LBO, SBO), id, (!first || j > 0) ? 1u : 0u);
                        mma_f16_ts(dtm, ah, sdesc(bl + off, LBO, SBO), id, 1u);
                        mma_f16_ts(dtm, al, sdesc(b0 + off, LBO, SBO), id, 1u);
                    }
                }
            };
            // a column-tile pair: one MMA of N = 256 per product into both
            // accumulators (2 x 128 columns, adjacent); B chunk of 256 rows
            // (hi plane, lo plane 16 KB on), K-major core matrices in the
            // pair packing's order (K step 8 KB apart) or, N = 64 pairs,
            // row-group-major (a row group's K core matrices contiguous)
            const uint32_t plbo = PP ? 128u : 2 * TBM * 16, psbo = PP ? uint32_t(8 * TBKR * 2) : SBO;
            const uint32_t pks = PP ? 256u : 4 * TBM * 16;  // bytes per K step of 16
            auto issue_pair = [&](uint32_t dtm, uint32_t a0, uint32_t b0, bool first) {
                const uint32_t id = idesc(1u, 2 * TBNR);
                const uint32_t bl = b0 + 2 * TBNR * TBKR * 2;
#pragma unroll
                for (int j = 0; j < TBKR / 16; ++j) {
                    const uint32_t off = uint32_t(j) * pks;
                    const uint32_t ah = a0 + uint32_t(16 * j), al = ah + 8u;
                    mma_f16_ts(dtm, ah, sdesc(b0 + off, plbo, psbo), id, (!first || j > 0) ? 1u : 0u);
                    mma_f16_ts(dtm, ah, sdesc(bl + off, plbo, psbo), id, 1u);
                    mma_f16_ts(dtm, al, sdesc(b0 + off, plbo, psbo), id, 1u);
                }
            };
            // the A operand of a chunk: TF32, the TMA slot; BF16x3, the TMEM stage
            auto a_of = [&](int rs, int tstage) {
                return PREC == 1 ? smem_u32(sm + C::OFF_RAW + rs * C::SLOT_RAW)
                                 : tmem + uint32_t(TM_A + tstage * TM_ASTAGE);
            };
            bool ok = true;
            if constexpr (BRES || BPACK) {
                int rs = 0, ts = 0;
                uint32_t rph = 0, tph = 0, u = 0;
                const int nts = BPACK ? nrs : NTS;
                int64_t gprev = -1;
                // packed B: the MMAs need no tile positions (a unit is nch
                // chunks of the rings whatever its tile)
                TileIter it;
                if (!BPACK && my_tiles > 0) it.start(d, mtiles, n_tiles, tblk, PP);
                for (int64_t l = 0; l < my_tiles && ok && !*abort_flag; l += TSTEP) {
                    int4 r = make_int4(0, 0, 0, 0);
                    int64_t g = 0;
                    if constexpr (!BPACK) {
                        r = it.record(d);
                        if (MODE != 2) g = it.f;
                        it.next(d, mtiles, n_tiles, tblk);
                    }
                    const int acc = int(l & (nacc - 1));  // pairs: acc 0 (and 1)
                    bool wok = true;
                    for (int t = 0; t < TSTEP; ++t)
                        wok = wok && mbar_wait(&X.tempty[acc + t], (uint32_t((l + t) >> nacc_sh) & 1u) ^ 1u);
                    if (!wok) {
                        ok = false;
                        break;
                    }
                    if (BRES && g != gprev) {  // new group: release the old B once its MMAs are done, wait for the new
                        if (u > 0) mma_commit(&X.bempty);
                        if (!mbar_wait(&X.bfull, u & 1u)) {
                            ok = false;
                            break;
                        }
                        ++u;
                        gprev = g;
                    }
                    tc_fence_after();
                    const uint32_t dtm = tmem + uint32_t(acc) * awr;
                    const int ctl = (MODE == 2 || d.sched != 0) ? 0 : r.w / TBN;  // the tile's column tile within the resident B
                    const uint32_t bset = smem_u32(sm + C::OFF_RAW + (nrs + ctl * nch) * C::SLOT_RAW);
                    for (int c = 0; c < nch; ++c) {
                        if (!mbar_wait(PREC == 2 ? &X.afull[ts] : &X.rfull[rs], PREC == 2 ? tph : rph)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t bch =
                            BPACK ? smem_u32(sm + C::OFF_RAW + (PAIR ? PAIR_ST + 2 * rs : PACK_ST + rs) * C::SLOT_RAW)
                                  : bset + c * C::SLOT_RAW;
                        if (PAIR)
                            issue_pair(dtm, a_of(rs, ts), bch, c == 0);
                        else
                            issue_chunk(dtm, a_of(rs, ts), bch, c == 0);
                        if (PREC == 2) mma_commit(&X.taempty[ts]);
                        if (PREC == 1 || BPACK) mma_commit(&X.rempty[rs]);
                        if (++rs == nrs) {
                            rs = 0;
                            rph ^= 1u;
                        }
                        if (++ts == nts) {
                            ts = 0;
                            tph ^= 1u;
                        }
                    }
                    if (ok)
                        for (int t = 0; t < TSTEP; ++t) mma_commit(&X.tfull[acc + t]);
                }
            } else {
                int64_t gch = 0;
                for (int64_t l = 0; l < my_tiles && ok && !*abort_flag; ++l) {
                    const int acc = int(l & (nacc - 1));
                    if (!mbar_wait(&X.tempty[acc], (uint32_t(l >> nacc_sh) & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dtm = tmem + uint32_t(acc) * awr;
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
                        issue_chunk(dtm, a_of(rs, slot), smem_u32(sm + C::OFF_B + slot * C::SLOT_B), c == 0);
                        mma_commit(&X.empty[slot]);
                        if (PREC == 1) mma_commit(&X.rempty[rs]);
                    }
                    if (ok) mma_commit(&X.tfull[acc]);
                }
            }
            if (!ok) give_up();
        }
        __syncwarp();
    } else if (warp == META_WARP) {
        // ------------------------------------------------------------ epilogue metadata
        // Per tile: the instance, rescale and exponent of each column, the
        // C base offset and the valid columns, into the slot ahead of the
        // epilogue.  The column data depend only on the tile's unit and
        // column tile, so they are loaded once per change (a unit spans
        // many row tiles) and kept in registers; the instance exponents E_C
        // are written here as well, once per instance: at its n = 0 column
        // in row tile 0.
        auto flush_max = [&](const EpiMeta &em) {
            if (!d.mxC) return;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c = lane + 32 * q;
                const uint32_t v = em.mx[c];
                if (v && em.inst[c] >= 0) record_max(d.mxC + em.inst[c], v);
            }
        };
        auto col_inst = [&](const int4 &r, int c) -> int {  // instance of tile column c, or -1
            const int64_t gc = int64_t(r.w) + c;
            return gc < (int64_t(r.y) << d.nb) ? r.x + int(gc >> d.nb) : -1;
        };
        TileIter it;
        if (my_tiles > 0) it.start(d, mtiles, n_tiles, tblk, PP);
        int64_t fprev = -1;
        int ctprev = -1;
        int inst_c[2] = {-1, -1}, ib_c[2] = {-1, -1}, eb_c[2] = {0, 0}, EB_c[2] = {0, 0};
        int ea_c = 0, EA_c = 0, ncv_c = 0, w_c = 0;
        int64_t base_c = 0;  // C offset of the tile's (row 0, column 0) with the row tile's bits left out
        bool ok = true;
        for (int64_t j = 0; j < my_tiles; ++j, it.next(d, mtiles, n_tiles, tblk)) {
            if (it.f != fprev || it.ct != ctprev) {
                const int4 r = it.record(d);
                const uint32_t mxa = d.mxA ? __ldg(d.mxA + r.z) : 0u;
                EA_c = __ldg(d.EA + r.z);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    inst_c[q] = col_inst(r, lane + 32 * q);
                    ib_c[q] = inst_c[q] >= 0 ? __ldg(d.instab + inst_c[q]).y : -1;
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    uint32_t mxb = 0u;
                    EB_c[q] = 0;
                    if (ib_c[q] >= 0) {
                        mxb = d.mxB ? __ldg(d.mxB + ib_c[q]) : 0u;
                        EB_c[q] = __ldg(d.EB + ib_c[q]);
                    }
                    eb_c[q] = d.mxB ? exp_of(mxb) : 0;
                }
                ea_c = d.mxA ? exp_of(mxa) : 0;
                const int64_t ncols = int64_t(r.y) << d.nb;
                ncv_c = int(ncols - r.w < TBN ? ncols - r.w : TBN);
                base_c = (int64_t(r.x) + (r.w >> d.nb)) * d.sC + dep(int64_t(r.w) & (N - 1), d.pCn, d.nb);
                w_c = r.w;
                fprev = it.f;
                ctprev = it.ct;
            }
            const int slot = int(j % MS);
            const bool w = mbar_wait(&X.mempty[slot], (uint32_t(j / MS) & 1u) ^ 1u);
            if (!__all_sync(0xffffffffu, w) || __any_sync(0xffffffffu, *abort_flag != 0)) {
                ok = false;
                break;
            }
            EpiMeta &em = X.epi[slot];
            // the slot's previous tile (j - MS) is done: its maxima go to
            // global memory from here, off the epilogue's path
            if (j >= MS) flush_max(em);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c = lane + 32 * q;
                const int inst = inst_c[q];
                em.inst[c] = inst;
                em.mx[c] = 0u;
                em.sc[c] = pow2f(-(ea_c + (MODE >= 2 ? 0 : eb_c[q])));  // dictionary and packed B carry 2^-eb
                if (MODE == 2) em.acol[c] = int16_t(inst >= 0 ? (ib_c[q] << d.nb) + ((w_c + c) & (N - 1)) : 0);
                if (inst >= 0 && it.mt == 0 && ((int64_t(w_c) + c) & (N - 1)) == 0)
                    d.EC[inst] = EA_c + ea_c + EB_c[q] + eb_c[q];
            }
            if (lane == 0) {
                em.base = base_c + dep(it.mt * TBM, d.pCm, d.mb);
                em.ncv = ncv_c;
            }
            mbar_arrive(&X.mfull[slot]);  // every lane (count 32): its writes are released
        }
        // flush the last MS tiles once the epilogue has released them
        for (int64_t j = my_tiles > MS ? my_tiles - MS : 0; ok && j < my_tiles; ++j) {
            const int slot = int(j % MS);
            const bool w = mbar_wait(&X.mempty[slot], uint32_t(j / MS) & 1u);
            if (!__all_sync(0xffffffffu, w)) {
                ok = false;
                break;
            }
            flush_max(X.epi[slot]);
        }
        if (!ok) give_up();
        __syncwarp();
    } else if (warp < EPI_WARP0 + NEPI / 32) {
        // ------------------------------------------------------------ epilogue
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(EPI_REGS));
        // Each warp drains 32 rows (its TMEM lane quadrant) x 16 complex
        // columns of each half tile: TMEM -> registers (max-|x| per
        // instance, power-of-two scale) -> its own 4 KB of shared memory in
        // destination order -> 16-byte stores, one contiguous run per
        // instruction where the C layout allows.  No barrier couples the
        // epilogue warps; the accumulator is released as soon as its last
        // half is in registers.
        const int ew = warp - EPI_WARP0;  // 0..7
        const int lanegrp = warp & 3;     // TMEM lanes 32*lanegrp ...
        const int sub = ew >> 2;          // 16-column block of a half
        const EpiMap &mp = X.map;
        uint8_t *wst = sm + C::OFF_STAGE + ew * 4096;
        // staging byte address of compressed index e: (swz(e >> 1) << 4) |
        // ((e & 1) << 3), linear over GF(2) in the bits of e; the row (lane)
        // and column bits of an element are disjoint, so its address is the
        // XOR of a per-lane part and a per-column part
        auto saddr = [](int ec) { return (stage_swz(ec >> 1) << 4) | ((ec & 1) << 3); };
        int erow = 0;  // compressed bits of this lane's row
#pragma unroll
        for (int b = 0; b < 5; ++b)
            if ((lane >> b) & 1) erow |= 1 << mp.rank[b];
        const int arow = saddr(erow);
        int acol[4];  // staging address parts of column bits 0-3
#pragma unroll
        for (int j = 0; j < 4; ++j) acol[j] = saddr(1 << mp.rank[5 + j]);
        const int alane = stage_swz(lane) << 4;  // store rounds read unit lane + 32 i
        int64_t offL = 0;  // compressed bits 1-5 = lane in the store rounds
        int colL = 0;
#pragma unroll
        for (int k = 1; k <= 5; ++k)
            if ((lane >> (k - 1)) & 1) {
                offL += mp.doff[k];
                colL += mp.dcol[k];
            }
        const int64_t doff0 = mp.doff[0];
        const int dcol0 = mp.dcol[0];
        const bool pair = mp.pair != 0;
        const bool rows_ok = lanegrp * 32 < mp.nrows;  // M = 64: quadrants 2 and 3 hold no rows
        const int64_t qoff = mp.qoff[lanegrp];
        const bool direct = mp.direct != 0;
        int64_t laneoff = 0;  // direct stores: C offset of this lane's row within its quadrant
#pragma unroll
        for (int b = 0; b < 5; ++b)
            if (b < d.mb && ((lane >> b) & 1)) laneoff += int64_t(1) << d.pCm[b];
        for (int64_t l = narrow ? sub : 0; l < my_tiles; l += narrow ? 2 : 1) {
            const int acc = int(l & (nacc - 1)), slot = int(l % MS);
            bool w = mbar_wait(&X.mfull[slot], uint32_t(l / MS) & 1u);
            w = w && mbar_wait(&X.tfull[acc], uint32_t(l >> nacc_sh) & 1u);
            if (!__all_sync(0xffffffffu, w) || __any_sync(0xffffffffu, *abort_flag != 0)) {
                give_up();
                break;
            }
            tc_fence_after();
            EpiMeta &em = X.epi[slot];
            const int ncv = em.ncv;
            const int nh = ncv > TBN / 2 ? 2 : 1;
            // halves of 8 columns this warp reads from the accumulator
            // (non-dictionary tiles of 8 columns: one)
            const int npass = (MODE != 2 && acw < 16) ? 1 : 2;
            for (int h = 0; h < nh; ++h) {
                const int c0 = narrow ? 0 : h * 32 + sub * 16;  // first column of this warp's block
                const bool act = rows_ok && c0 < ncv;  // warp-uniform
                // the block's complex columns (16, or 8 where no tile has
                // more: NC), every load issued before one wait
                auto block = [&](auto nc_) {
                    constexpr int NC = decltype(nc_)::value;
                    uint32_t r[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) r[q] = 0u;
                    if (act && MODE == 2) {
                        const uint32_t tb = tmem + uint32_t(acc) * awr + (uint32_t(lanegrp * 32) << 16);
                        switch (N < NC ? N : NC) {
                            case 1: tmem_gather16<NC, 1>(r, tb, em, c0, ncv); break;
                            case 2: tmem_gather16<NC, 2>(r, tb, em, c0, ncv); break;
                            case 4: tmem_gather16<NC, 4>(r, tb, em, c0, ncv); break;
                            case 8: tmem_gather16<NC, 8>(r, tb, em, c0, ncv); break;
                            default: tmem_gather16<NC, NC>(r, tb, em, c0, ncv); break;
                        }
                    } else if (act) {
                        const uint32_t ta =
                            tmem + uint32_t(acc) * awr + uint32_t(c0 * 2) + (uint32_t(lanegrp * 32) << 16);
                        if (NC == 16 && npass == 2) tmem_ld<16>(ta + 16u, r + 16);
                        tmem_ld<16>(ta, r);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    }
                    if (h == nh - 1) {  // the accumulator is free for a later tile
                        tc_fence_before();
                        mbar_arrive(&X.tempty[acc]);
                    }
                    if (!act) return;
                    if (d.mxC) {
                        switch (N < NC ? N : NC) {
                            case 1: fold_max16<NC, 1, MODE == 1>(r, em, c0, lane); break;
                            case 2: fold_max16<NC, 2, MODE == 1>(r, em, c0, lane); break;
                            case 4: fold_max16<NC, 4, MODE == 1>(r, em, c0, lane); break;
                            case 8: fold_max16<NC, 8, MODE == 1>(r, em, c0, lane); break;
                            default: fold_max16<NC, NC, MODE == 1>(r, em, c0, lane); break;
                        }
                    }
                    if (NC == 8 && direct) {
                        // each lane its row's valid columns, straight from registers
                        float2 *rowp = d.C + (em.base + qoff + laneoff);
#pragma unroll
                        for (int jj = 0; jj < NC; ++jj) {
                            if (jj >= ncv) break;
                            const float sv = MODE == 1 ? 1.f : em.sc[jj];
                            rowp[mp.coff[jj]] =
                                make_float2(__uint_as_float(r[2 * jj]) * sv, __uint_as_float(r[2 * jj + 1]) * sv);
                        }
                        return;
                    }
                    // scale and stage in destination order
#pragma unroll
                    for (int q = 0; q < NC / 4; ++q) {
                        const float4 sc4 = *reinterpret_cast<const float4 *>(&em.sc[c0 + 4 * q]);
                        const float scq[4] = {sc4.x, sc4.y, sc4.z, sc4.w};
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int jj = 4 * q + t;  // column within the warp's block
                            int a = arow;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if ((jj >> j) & 1) a ^= acol[j];
                            // resident B carries the rescale already
                            const float sv = MODE == 1 ? 1.f : scq[t];
                            *reinterpret_cast<float2 *>(wst + a) =
                                make_float2(__uint_as_float(r[2 * jj]) * sv, __uint_as_float(r[2 * jj + 1]) * sv);
                        }
                    }
                };
                if (ow <= 8)
                    block(std::integral_constant<int, 8>());
                else
                    block(std::integral_constant<int, 16>());
                if (!act || direct) continue;
                const int ncw = ncv - c0;  // valid columns of this block
                __syncwarp();
                const int64_t wb = em.base + qoff + mp.hoff[narrow ? 0 : h * 2 + sub] + offL;
                if (pair && ncw >= 16) {  // whole block valid, 16-byte runs: straight-line stores
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 val = *reinterpret_cast<const float4 *>(wst + (alane ^ (stage_swz(32 * i) << 4)));
                        *reinterpret_cast<float4 *>(d.C + (wb + mp.offI[i])) = val;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        // compressed elements 2u, 2u + 1 with u = lane + 32 i
                        const float4 val = *reinterpret_cast<const float4 *>(wst + (alane ^ (stage_swz(32 * i) << 4)));
                        const int c = colL + mp.colI[i];
                        const bool v0 = c < ncw, v1 = c + dcol0 < ncw;
                        float2 *dst = d.C + (wb + mp.offI[i]);
                        if (pair && v0 && v1) {
                            *reinterpret_cast<float4 *>(dst) = val;
                        } else {
                            if (v0) dst[0] = make_float2(val.x, val.y);
                            if (v1) dst[doff0] = make_float2(val.z, val.w);
                        }
                    }
                }
                __syncwarp();  // the staging area is rewritten by the next half
            }
            mbar_arrive(&X.mempty[slot]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_alloc_cols<PREC>()) : "memory");
    }
}

// Packed B (MODE 3): every B instance of the step, 64 columns x 16 complex
// k per 16 KB block (block (ib * N/64 + column tile) * nch + chunk) in the
// layout of a B stage (real 2x2 form, K-major, TF32 or BF16 hi and lo
// planes), each column multiplied by its instance's 2^-eb (exact).  One
// block per CTA; thread (column, k quad) as in the producers' expansion.
// RM: row-group-major order (N = 64 column-tile pairs: two instances'
// blocks side by side form one operand of 256 rows).
template <int PREC, bool RM = false>
__global__ void __launch_bounds__(256) k_pack_b(const StepDesc d, int nch) {
    const int tid = threadIdx.x, bcol = tid & 63, kqb = tid >> 6;
    const int64_t blk = blockIdx.x;
    const int c = int(blk % nch);
    const int64_t ct_all = blk / nch;  // ib * (N / 64) + column tile
    const int64_t ib = ct_all >> (d.nb - 6);
    const int64_t n = ((ct_all & ((int64_t(1) << (d.nb - 6)) - 1)) << 6) + bcol;
    const int K = 1 << d.kb;
    const int k = c * TBK + 4 * kqb;
    const float s = d.mxB ? pow2f(-exp_of(__ldg(d.mxB + ib))) : 1.f;
    float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
    if (k + 3 < K) {
        const float4 *src = reinterpret_cast<const float4 *>(d.B + ib * d.sB + (n << d.kb) + k);
        p0 = __ldg(src);
        p1 = __ldg(src + 1);
    }
    expand_b<PREC, RM>(d.bpack + blk * (TBNR * TBKR * 4), bcol, kqb,
                   make_float4(p0.x * s, p0.y * s, p0.z * s, p0.w * s),
                   make_float4(p1.x * s, p1.y * s, p1.z * s, p1.w * s));
}

// Packed B for column-tile pairs (MODE 4): 128 columns x 16 complex k per
// 32 KB block (block (ib * N/128 + pair) * nch + chunk) in the layout of a
// B operand of 256 rows; thread (column, k quad) expands columns c and
// c + 64 of its pair.
template <int PREC>
__global__ void __launch_bounds__(256) k_pack_b_pair(const StepDesc d, int nch) {
    const int tid = threadIdx.x, bcol = tid & 63, kqb = tid >> 6;
    const int64_t blk = blockIdx.x;
    const int c = int(blk % nch);
    const int64_t cp_all = blk / nch;  // ib * (N / 128) + pair
    const int64_t ib = cp_all >> (d.nb - 7);
    const int64_t n0 = (cp_all & ((int64_t(1) << (d.nb - 7)) - 1)) << 7;
    const int K = 1 << d.kb;
    const int k = c * TBK + 4 * kqb;
    const float s = d.mxB ? pow2f(-exp_of(__ldg(d.mxB + ib))) : 1.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
        if (k + 3 < K) {
            const float4 *src = reinterpret_cast<const float4 *>(d.B + ib * d.sB + ((n0 + 64 * h + bcol) << d.kb) + k);
            p0 = __ldg(src);
            p1 = __ldg(src + 1);
        }
        expand_b<PREC>(d.bpack + blk * (2 * TBNR * TBKR * 4), bcol + 64 * h, kqb,
                       make_float4(p0.x * s, p0.y * s, p0.z * s, p0.w * s),
                       make_float4(p1.x * s, p1.y * s, p1.z * s, p1.w * s), 2 * TBNR);
    }
}

}  // namespace

int64_t tc_packed_b_bytes(const StepDesc &d) {
    if (d.nb < 6 || !gemm_tc_supports(d)) return 0;
    const int64_t nch = ((int64_t(1) << d.kb) + TBK - 1) / TBK;
    return d.nInstB * (int64_t(1) << (d.nb - 6)) * nch * int64_t(TBNR * TBKR * 4);
}

bool gemm_tc_supports(const StepDesc &d) {
    // K >= 8 complex (at least half a chunk), 64 <= M < 2^31 rows
    return d.kb >= 3 && d.mb >= 6 && d.mb <= 30 && d.kb <= 24;
}

int tc_dictionary_chunks(const StepDesc &d) {
    // schedule 0 with every B instance of the step in one 64-column tile
    // (and K within the pool): the B dictionary's chunk count, else 0
    if (!d.tc_resident_b || d.sched != 0 || (d.nInstB << d.nb) > TBN) return 0;
    const int64_t nch = ((int64_t(1) << d.kb) + TBK - 1) / TBK;
    return nch <= BRES_MAX_B ? int(nch) : 0;
}

int tc_resident_b_chunks(const StepDesc &d) {
    // B chunks resident at a time: schedule 0, the largest group's (its
    // 64-column tiles x K chunks); schedule 1, one column tile's; 0 when they
    // do not fit the resident-B pool
    if (!d.tc_resident_b) return 0;
    const int64_t nch = ((int64_t(1) << d.kb) + TBK - 1) / TBK;
    const int64_t nct = d.sched != 0 ? 1 : ((int64_t(d.max_group) << d.nb) + TBN - 1) / TBN;
    const int64_t n = nch * nct;
    return n >= 1 && n <= BRES_MAX_B ? int(n) : 0;
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
    e = cudaFuncSetAttribute(reinterpret_cast<const void *>(k_step_gemm_tc<2, 4>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<2, true>());
    if (e != cudaSuccess) return e;
    const void *fns[8] = {reinterpret_cast<const void *>(k_step_gemm_tc<1, 0>),
                          reinterpret_cast<const void *>(k_step_gemm_tc<2, 0>),
                          reinterpret_cast<const void *>(k_step_gemm_tc<1, 1>),
                          reinterpret_cast<const void *>(k_step_gemm_tc<2, 1>),
                          reinterpret_cast<const void *>(k_step_gemm_tc<1, 2>),
                          reinterpret_cast<const void *>(k_step_gemm_tc<2, 2>),
                          reinterpret_cast<const void *>(k_step_gemm_tc<1, 3>),
                          reinterpret_cast<const void *>(k_step_gemm_tc<2, 3>)};
    const int bytes[8] = {(int)smem_bytes<1, false>(), (int)smem_bytes<2, false>(), (int)smem_bytes<1, true>(),
                          (int)smem_bytes<2, true>(),  (int)smem_bytes<1, true>(),  (int)smem_bytes<2, true>(),
                          (int)smem_bytes<1, true>(),  (int)smem_bytes<2, true>()};
    for (int i = 0; i < 8; ++i) {
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The A operand of a step as a 3-D tensor for TMA: (real k = 2K floats of a
// row, rows m, instances).  The box (32, 128, 1) lands in shared memory as
// 128 rows of 128 bytes with the 128-byte swizzle, the K-major layout the
// MMA descriptors use; each load is 128 row segments of 128 contiguous
// bytes.  Rows past M and k past K read as zeros.
cudaError_t make_a_map(const StepDesc &d, int64_t n_inst_a, CUtensorMap *map) {
    if (!g_encode) return cudaErrorNotReady;
    const cuuint64_t K = cuuint64_t(1) << d.kb;
    const cuuint64_t dims[3] = {2 * K, cuuint64_t(1) << d.mb, cuuint64_t(n_inst_a)};
    const cuuint64_t strides[2] = {K * 8, cuuint64_t(d.sA) * 8};
    const cuuint32_t box[3] = {TBKR, TBM, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(d.A), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
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
    const dim3 g((unsigned)grid);
    // B as a dictionary (every instance resident for the launch), else
    // resident per group or column tile when it fits the pool, else streamed
    const int ndict = tc_dictionary_chunks(d);
    const int nbset = ndict > 0 ? ndict : tc_resident_b_chunks(d);
    const int nrs = std::min(Cfg<2, true>::RST, Cfg<2, true>::NSLOT - nbset);
    // accumulator and output widths (complex columns, powers of two in
    // [8, 64]): the most columns a tile has, or the dictionary's width
    auto width = [](int64_t cols) {
        int w = 8;
        while (w < cols && w < TBN) w <<= 1;
        return w;
    };
    const int ow = width(int64_t(d.max_group) << d.nb);
    const int acw = ndict > 0 ? width(d.nInstB << d.nb) : ow;
    // B streamed or packed (not held per unit): blocks of tiles dealt
    // round-robin, each block the tiles that share one operand tile
    // (schedule 1: a column tile's row tiles; schedule 0: a row tile's
    // column tiles), so that the operands the CTAs read at any time fit L2
    auto block_of = [&]() -> int {
        const int64_t b = d.sched != 0 ? mtiles : ((int64_t(d.max_group) << d.nb) + TBN - 1) / TBN;
        return (b >= 1 && b * grid * 2 <= tiles) ? int(b) : 0;
    };
    // B packed once per launch in MMA form and streamed from L2 where it is
    // neither a dictionary nor resident and N >= 64 (a tile's columns lie
    // in one B instance), if the plan reserved room for it
    const int64_t pack = tc_packed_b_bytes(d);
    const int nch_all = int(((int64_t(1) << d.kb) + TBK - 1) / TBK);
    // a resident B whose unit (schedule 1: a column tile, 0: a group) runs
    // fewer than 64 chunks is packed instead where it can be: its load does
    // not overlap the MMAs, and the unit's MMAs would not hide it
    const int64_t unit_chunks =
        (d.sched != 0 ? mtiles : mtiles * (((int64_t(d.max_group) << d.nb) + TBN - 1) / TBN)) * nch_all;
    if (ndict == 0 && (nbset == 0 || unit_chunks < 64) && d.tc_resident_b && pack > 0 && d.bpack &&
        pack <= d.bpack_bytes) {
        const int nch = int(((int64_t(1) << d.kb) + TBK - 1) / TBK);
        const int64_t blocks = pack / (TBNR * TBKR * 4);
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        // BF16x3, schedule 0, N >= 64: column tiles in pairs (a row tile's
        // consecutive tiles; N >= 128 gives every group an even count, with
        // N = 64 groups of odd size get a pad tile), one MMA of N = 256 for
        // both; the pairs dealt round-robin one at a time, so that the CTAs
        // walking one row tile's pairs run side by side and read its A from
        // L2 (blocks of the whole row tile per CTA re-read A from DRAM once
        // per pair: 10 % slower on 2^12 x 2^9 x 2^8); N = 64 only where pad
        // tiles add at most 1/8 (groups of one instance would double the
        // MMAs).  K >= 256 only: a pair holds both accumulators, so its
        // epilogue does not overlap the next pair's MMAs, which costs more
        // than the halved MMA issue gains on short K (measured: K = 128
        // 5-12 % slower, K = 256 1-10 % faster, K = 512 22-49 % faster)
        const bool pad_ok = d.nb == 6 && d.ptab && d.n_ptab * 8 <= d.n_ctab * 9;
        if (precision == 2 && d.sched == 0 && d.kb >= 8 && (d.nb >= 7 || pad_ok) && d.tc_pair) {
            if (d.nb == 6)
                k_pack_b<2, true><<<dim3((unsigned)blocks), 256, 0, s>>>(d, nch);
            else
                k_pack_b_pair<2><<<dim3((unsigned)(blocks / 2)), 256, 0, s>>>(d, nch);
            k_step_gemm_tc<2, 4><<<g, NTHREADS, smem_bytes<2, true>(), s>>>(d, mtiles, err, *a_map, PAIR_ST, acw, ow, 2);
            return cudaGetLastError();
        }
        if (precision == 1) {
            k_pack_b<1><<<dim3((unsigned)blocks), 256, 0, s>>>(d, nch);
            k_step_gemm_tc<1, 3><<<g, NTHREADS, smem_bytes<1, true>(), s>>>(d, mtiles, err, *a_map, PACK_ST, acw, ow,
                                                                            block_of());
        } else {
            k_pack_b<2><<<dim3((unsigned)blocks), 256, 0, s>>>(d, nch);
            k_step_gemm_tc<2, 3><<<g, NTHREADS, smem_bytes<2, true>(), s>>>(d, mtiles, err, *a_map, PACK_ST, acw, ow,
                                                                            block_of());
        }
        return cudaGetLastError();
    }
    if (ndict > 0) {
        if (precision == 1)
            k_step_gemm_tc<1, 2><<<g, NTHREADS, smem_bytes<1, true>(), s>>>(d, mtiles, err, *a_map, nrs, acw, ow, 0);
        else
            k_step_gemm_tc<2, 2><<<g, NTHREADS, smem_bytes<2, true>(), s>>>(d, mtiles, err, *a_map, nrs, acw, ow, 0);
    } else if (nbset > 0) {
        if (precision == 1)
            k_step_gemm_tc<1, 1><<<g, NTHREADS, smem_bytes<1, true>(), s>>>(d, mtiles, err, *a_map, nrs, acw, ow, 0);
        else
            k_step_gemm_tc<2, 1><<<g, NTHREADS, smem_bytes<2, true>(), s>>>(d, mtiles, err, *a_map, nrs, acw, ow, 0);
    } else if (precision == 1) {
        k_step_gemm_tc<1, 0><<<g, NTHREADS, smem_bytes<1, false>(), s>>>(d, mtiles, err, *a_map, Cfg<1, false>::RST,
                                                                         acw, ow, block_of());
    } else {
        k_step_gemm_tc<2, 0><<<g, NTHREADS, smem_bytes<2, false>(), s>>>(d, mtiles, err, *a_map, Cfg<2, false>::RST,
                                                                         acw, ow, block_of());
    }
    return cudaGetLastError();
}

}  // namespace tnk
