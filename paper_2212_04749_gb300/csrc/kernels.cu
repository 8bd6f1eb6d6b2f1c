// CUDA-core kernels of the contraction path (sm_103a).
//
//   k_fill           leaf instance blocks for one slice batch (the fused gate
//                    tensors with output legs projected on the bitstrings'
//                    values and sliced legs on the slice's values)
//   k_step_row       one pairwise step C = A (x) B with a small B operand
//                    (N <= 16, K*N <= 256), grouped by shared A instance: each
//                    A row is read once and multiplied by every B block of
//                    its group; the bandwidth-bound "high-rank x low-rank"
//                    contraction of SM Sec. V.A
//   k_step_gemm_simt tiled complex GEMM with gathered (bit-permuted) operand
//                    loads, FP32 FMA; the plain FP32 form of big x big steps
//   k_accumulate     amp[p] += sum over the batch's slices of the root
//                    partials times 2^E, complex128, fixed slice order
//                    (first-level slicing, SM Sec. IV.B)
//   k_xeb            FP64 fixed-order reduction of sum |amp|^2 (Eq. fxeb)
//   k_pt_moments     FP64 sums for the Porter-Thomas mixture fit of the
//                    fidelity (density of Eq. fxeb) and the linear XEB's error
//   k_pt_hist        histogram of x = N |amp|^2 (integer counts)
//   k_sample         one completion per correlated batch, drawn with
//                    probability |amp|^2 / sum over the batch (perfect
//                    sample from a batch, main text on Fig. 3(b), SM Sec. II)
//
// Power-of-two rescaling: every produced instance records the largest
// |component| of its entries (as float bits, atomicMax of non-negative
// floats); its consumer multiplies the loaded values by 2^-e, e the
// exponent of that maximum, and adds e to the output's exponent E.  Scaling
// by a power of two is exact, so with and without it the FP32 results are
// bitwise the same (barring subnormals).
#include "kernels.cuh"

namespace tnk {

namespace {

__device__ __forceinline__ int exp_of(uint32_t bits) {
    if (bits == 0u) return 0;
    int e = int((bits >> 23) & 0xffu) - 127;
    return max(-126, min(126, e));
}

__device__ __forceinline__ float pow2f(int e) {  // 2^e, |e| <= 126
    return __int_as_float((127 + e) << 23);
}

__device__ __forceinline__ uint32_t absmax_bits(float2 v) {
    return __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y)));
}

__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

__device__ __forceinline__ int64_t dep(int64_t x, const int8_t *pos, int nbits) {
    int64_t r = 0;
    for (int j = 0; j < nbits; ++j) r |= ((x >> j) & 1) << pos[j];
    return r;
}

// raise the recorded maximum only when it grows (monotone, so the
// unsynchronised read is safe)
// fire-and-forget global max (a reduction, no returned value: the issuing
// thread never waits on memory)
__device__ __forceinline__ void record_max(uint32_t *slot, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(slot), "r"(v) : "memory");
}

__global__ void k_fill(const FillJobD *__restrict__ jobs, int64_t njobs, const LeafHighD *__restrict__ highs,
                       int64_t batch, float2 *__restrict__ ws) {
    const int64_t job = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (job >= njobs) return;
    const FillJobD J = jobs[job];
    const LeafHighD H = highs[J.leaf_high];
    int64_t src = J.src;
    for (int c = 0; c < H.cnt; ++c) src += ((batch >> H.j[c]) & 1) * int64_t(H.stride[c]);
    for (int e = lane; e < J.n; e += 32) ws[J.dst + e] = ws[src + e];
}

constexpr int ROW_THREADS = 256;
constexpr int ROW_SB = 2048;  // staged B entries (complex) per block: 16 KB
constexpr int ROW_CH = 32;    // most instances staged at once

// Small-rank step (N = 2^NB <= 16, K*N <= 256), grouped: the output
// instances that read one A instance (a group) are computed together, so
// every A row is read once and multiplied by each of the group's B blocks.
// A row's K-contiguous run (rows are affine: A + m*K) is split over
// L = min(8, K/2) lanes holding KL = K/L complex values each in registers,
// loaded 16 bytes at a time; each output's partial products are summed over
// the row's L lanes with xor-shuffles.  R = 32/L rows per warp pass.
//   uniform (M >= 8R): a block = rows_per_block rows of one group; the
//     group's B blocks (column-affine: K*N contiguous complex each) are
//     staged in shared memory, ROW_SB entries at a time; max-|x| words and
//     exponents are recorded once per instance.
//   small instances (M < 8R): a block = rows_per_block consecutive rows of
//     consecutive groups, each row looping over its group's instances; B
//     comes through the L1 cache.  Schedule 1: rows_per_block consecutive
//     (instance, row) pairs, one per lane group, so that the instances of
//     large groups run in parallel.
template <int NB, int KL>
__global__ void __launch_bounds__(ROW_THREADS) k_step_row(const StepDesc d, int rows_per_block, int64_t mblocks) {
    constexpr int N = 1 << NB;
    __shared__ int8_t s_pCm[40];
    __shared__ int64_t s_offCn[N];
    __shared__ int64_t s_mloC[256];
    __shared__ __align__(16) float2 s_B[ROW_SB];
    __shared__ int64_t s_ib[ROW_CH];
    __shared__ int32_t s_e[ROW_CH], s_EC[ROW_CH];
    __shared__ uint32_t s_mx[ROW_CH];
    __shared__ int64_t s_pass_off[16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = 1 << d.kb;
    const int KN = K * N;
    const int mb = d.mb;
    const int64_t M = int64_t(1) << mb;
    const int L = K / KL;  // lanes per row (row_lanes on the host)
    const int R = 32 / L;
    const int sub = lane / L, kl = lane % L;
    const int passes = rows_per_block / (8 * R);
    if (tid < 40) s_pCm[tid] = d.pCm[tid];
    if (tid < N) s_offCn[tid] = dep(tid, d.pCn, NB);
    __syncthreads();
    {
        const int lob = mb < 8 ? mb : 8;
        s_mloC[tid] = dep(tid & ((1 << lob) - 1), s_pCm, lob);
    }
    __syncthreads();

    // this lane's KL values of row m of A instance ia
    auto load_row = [&](float2 (&a)[KL], int64_t ia, int64_t m, bool valid) {
        const float2 *A = d.A + ia * d.sA + (m << d.kb);
        if (KL == 1) {
            a[0] = valid ? __ldg(A) : make_float2(0.f, 0.f);
        } else {
#pragma unroll
            for (int q = 0; q < KL / 2; ++q) {
                const float4 v = valid ? __ldg(reinterpret_cast<const float4 *>(A + 2 * kl + 2 * L * q))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                a[2 * q] = make_float2(v.x, v.y);
                a[2 * q + 1] = make_float2(v.z, v.w);
            }
        }
    };
    // acc[n] = sum over this lane's k of a[k] B[n*K + k], then summed over
    // the row's L lanes by recursive halving: at xor level o = 1, 2, 4 a lane
    // keeps one half of the outputs it still holds (the upper half when bit o
    // of its lane index is set) and adds its partner's copy of that half;
    // once one output is left, plain xor sums finish.  Afterwards each lane
    // holds max(1, N / L) outputs (n0, n_held below).
    auto row_times_b = [&](float2 (&acc)[N], const float2 (&a)[KL], const float2 *Bj) {
#pragma unroll
        for (int n = 0; n < N; ++n) acc[n] = make_float2(0.f, 0.f);
        if (KL == 1) {
#pragma unroll
            for (int n = 0; n < N; ++n) cfma(acc[n], a[0], Bj[n * K]);
        } else {
#pragma unroll
            for (int q = 0; q < KL / 2; ++q) {
                const int k = 2 * kl + 2 * L * q;
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    const float4 b = *reinterpret_cast<const float4 *>(Bj + n * K + k);
                    cfma(acc[n], a[2 * q], make_float2(b.x, b.y));
                    cfma(acc[n], a[2 * q + 1], make_float2(b.z, b.w));
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int o = 1 << t;
            if (o >= L) break;
            constexpr int W0 = N;
            const int width = W0 >> t;  // a constant once unrolled
            if (width > 1) {
                const bool up = (kl & o) != 0;
#pragma unroll
                for (int n = 0; n < N / 2; ++n) {
                    if (n < (width >> 1)) {
                        const int h = width >> 1;
                        const float2 send = up ? acc[n] : acc[n + h];
                        const float2 keep = up ? acc[n + h] : acc[n];
                        acc[n].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, o);
                        acc[n].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, o);
                    }
                }
            } else {
                acc[0].x += __shfl_xor_sync(0xffffffffu, acc[0].x, o);
                acc[0].y += __shfl_xor_sync(0xffffffffu, acc[0].y, o);
            }
        }
    };
    // outputs this lane holds after row_times_b: acc[j] is output n0 + j
    int n0 = 0, n_held = N;
    for (int t = 0; (1 << t) < L && n_held > 1; ++t) {
        n_held >>= 1;
        if (kl & (1 << t)) n0 += n_held;
    }
    const bool store_lane = N >= L || kl < N;  // higher lane bits hold copies

    if (M >= 8 * R) {
        const int64_t g = int64_t(blockIdx.x) / mblocks;
        const int64_t m0 = (int64_t(blockIdx.x) - g * mblocks) * rows_per_block;
        const int64_t i0 = d.gfirst[g], cnt = d.gfirst[g + 1] - i0;
        const int64_t ia = d.instab[i0].x;
        const int ea = d.mxA ? exp_of(d.mxA[ia]) : 0;
        const int EAa = d.EA[ia] + ea;
        const int ch_max = min(ROW_CH, ROW_SB / KN);
        for (int64_t c0 = 0; c0 < cnt; c0 += ch_max) {
            const int ch = int(cnt - c0 < ch_max ? cnt - c0 : int64_t(ch_max));
            if (tid < ch) {
                const int64_t ib = d.instab[i0 + c0 + tid].y;
                const int eb = d.mxB ? exp_of(d.mxB[ib]) : 0;
                s_ib[tid] = ib;
                s_e[tid] = ea + eb;
                s_EC[tid] = EAa + d.EB[ib] + eb;
                s_mx[tid] = 0u;
            }
            if (tid < passes) s_pass_off[tid] = dep(int64_t(tid) * 8 * R, s_pCm, mb);
            __syncthreads();
            // B staged with each instance's power-of-two rescale folded in (exact)
            for (int e = tid; e < ch * KN; e += ROW_THREADS) {
                const int j = e / KN;
                const float sc = pow2f(-s_e[j]);
                const float2 b = __ldg(d.B + s_ib[j] * d.sB + (e - j * KN));
                s_B[e] = make_float2(b.x * sc, b.y * sc);
            }
            __syncthreads();
            // row m = m0 + it 8R + (warp R + sub): three disjoint bit ranges,
            // so its C offset is this lane's part plus the pass's part
            const int64_t lane_off = dep(m0 + int64_t(warp) * R + sub, s_pCm, mb);
            // max-|x| per instance: in registers across the passes when the
            // chunk has at most 4 instances, reduced over the warp once
            const bool few = ch <= 4;
            uint32_t mxr[4] = {0u, 0u, 0u, 0u};
            // the next pass's A row is loaded while this pass computes
            float2 a_nx[KL];
            load_row(a_nx, ia, m0 + int64_t(warp) * R + sub, true);
            for (int it = 0; it < passes; ++it) {
                float2 a[KL];
#pragma unroll
                for (int q = 0; q < KL; ++q) a[q] = a_nx[q];
                if (it + 1 < passes) load_row(a_nx, ia, m0 + (int64_t(it + 1) * 8 + warp) * R + sub, true);
                const int64_t offC = lane_off + s_pass_off[it];
                for (int j = 0; j < ch; ++j) {
                    float2 acc[N];
                    row_times_b(acc, a, s_B + j * KN);
                    float2 *C = d.C + (i0 + c0 + j) * d.sC + offC;
                    uint32_t mx = 0;
                    if (store_lane) {
#pragma unroll
                        for (int h = 0; h < N; ++h) {
                            if (h >= n_held) break;
                            C[s_offCn[n0 + h]] = acc[h];
                            mx = max(mx, absmax_bits(acc[h]));
                        }
                    }
                    if (d.mxC) {
                        if (few) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                if (q == j) mxr[q] = max(mxr[q], mx);
                        } else {
                            const uint32_t r = __reduce_max_sync(0xffffffffu, mx);
                            if (lane == 0 && r) atomicMax(&s_mx[j], r);
                        }
                    }
                }
            }
            if (d.mxC && few) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q >= ch) break;
                    const uint32_t r = __reduce_max_sync(0xffffffffu, mxr[q]);
                    if (lane == 0 && r) atomicMax(&s_mx[q], r);
                }
            }
            __syncthreads();
            if (tid < ch) {
                const int64_t i = i0 + c0 + tid;
                if (m0 == 0) d.EC[i] = s_EC[tid];
                if (d.mxC && s_mx[tid]) record_max(d.mxC + i, s_mx[tid]);
            }
            __syncthreads();
        }
    } else if (d.sched == 1) {
        // small instances, schedule 1: one output instance row per lane
        // group (instances of large groups run in parallel; their shared A
        // rows come through the caches)
        const int64_t total = d.nInst << mb;
        for (int it = 0; it < passes; ++it) {
            const int64_t gid = int64_t(blockIdx.x) * rows_per_block + (int64_t(it) * 8 + warp) * R + sub;
            const bool valid = gid < total;
            const int64_t gr = valid ? gid : 0;
            const int64_t i = gr >> mb, m = gr & (M - 1);
            const int2 ab = d.instab[i];
            const int ea = d.mxA ? exp_of(d.mxA[ab.x]) : 0;
            const int eb = d.mxB ? exp_of(d.mxB[ab.y]) : 0;
            float2 a[KL];
            load_row(a, ab.x, m, valid);
            float2 acc[N];
            row_times_b(acc, a, d.B + int64_t(ab.y) * d.sB);
            const float sc = pow2f(-(ea + eb));
            uint32_t mx = 0;
            if (valid) {
                float2 *C = d.C + i * d.sC + (mb > 8 ? dep(m >> 8, s_pCm + 8, mb - 8) : 0) + s_mloC[m & 255];
                if (store_lane) {
#pragma unroll
                    for (int h = 0; h < N; ++h) {
                        if (h >= n_held) break;
                        const float2 v = make_float2(acc[h].x * sc, acc[h].y * sc);
                        C[s_offCn[n0 + h]] = v;
                        mx = max(mx, absmax_bits(v));
                    }
                }
                if (m == 0 && kl == 0) d.EC[i] = d.EA[ab.x] + ea + d.EB[ab.y] + eb;
            }
            for (int o = L >> 1; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (d.mxC && valid && kl == 0 && mx) record_max(d.mxC + i, mx);
        }
    } else {
        const int64_t total = d.n_groups << mb;
        for (int it = 0; it < passes; ++it) {
            const int64_t gid = int64_t(blockIdx.x) * rows_per_block + (int64_t(it) * 8 + warp) * R + sub;
            const bool valid = gid < total;
            const int64_t gr = valid ? gid : 0;
            const int64_t g = gr >> mb, m = gr & (M - 1);
            const int64_t i0 = d.gfirst[g];
            const int cnt = valid ? int(d.gfirst[g + 1] - i0) : 0;
            const int64_t ia = d.instab[i0].x;
            const int ea = d.mxA ? exp_of(d.mxA[ia]) : 0;
            float2 a[KL];
            load_row(a, ia, m, valid);
            const int64_t offC = (mb > 8 ? dep(m >> 8, s_pCm + 8, mb - 8) : 0) + s_mloC[m & 255];
            const int jmax = int(__reduce_max_sync(0xffffffffu, uint32_t(cnt)));  // warp-uniform trip count
            for (int j = 0; j < jmax; ++j) {
                const bool vj = j < cnt;
                const int64_t i = i0 + j;
                const int64_t ib = vj ? d.instab[i].y : 0;
                float2 acc[N];
                row_times_b(acc, a, d.B + ib * d.sB);
                const int eb = vj && d.mxB ? exp_of(d.mxB[ib]) : 0;
                const float sc = pow2f(-(ea + eb));
                uint32_t mx = 0;
                if (vj) {
                    float2 *C = d.C + i * d.sC + offC;
                    if (store_lane) {
#pragma unroll
                        for (int h = 0; h < N; ++h) {
                            if (h >= n_held) break;
                            const float2 v = make_float2(acc[h].x * sc, acc[h].y * sc);
                            C[s_offCn[n0 + h]] = v;
                            mx = max(mx, absmax_bits(v));
                        }
                    }
                    if (m == 0 && kl == 0) d.EC[i] = d.EA[ia] + ea + d.EB[ib] + eb;
                }
                for (int o = L >> 1; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (d.mxC && vj && kl == 0 && mx) record_max(d.mxC + i, mx);
            }
        }
    }
}

// Grouped SIMT complex GEMM, FP32 FMA.  One CTA: BM rows of the group's A
// instance times BN columns of the group's concatenated B instances (column
// c -> instance gfirst[g] + c / N, column n = c % N), K in chunks of BK.
// 256 threads, 8 x 4 outputs each (rows tm + 16 x, columns 4 tn + y).
constexpr int GBM = 128, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) k_step_gemm_simt(const StepDesc d, int ctiles, int mtiles) {
    __shared__ int8_t s_pAm[40], s_pCm[40];
    __shared__ int64_t s_offA[GBM], s_offC[GBM];
    __shared__ int64_t s_bbase[GBN], s_cbase[GBN];
    __shared__ int32_t s_eb[GBN];
    __shared__ uint32_t s_mx[GBN];
    __shared__ float2 s_A[GBK][GBM + 2];
    __shared__ float2 s_B[GBK][GBN + 2];
    __shared__ int64_t s_ia;
    __shared__ int s_ea;
    const int tid = threadIdx.x;
    const int64_t bid = blockIdx.x;
    // schedule 0: row tiles of a column tile on consecutive blocks (the
    // group's B columns stay in L2); 1: column tiles of a row tile on
    // consecutive blocks (the A rows stay in L2)
    int mt, ct;
    int64_t g;
    if (d.sched == 0) {
        mt = int(bid % mtiles);
        const int64_t rest = bid / mtiles;
        ct = int(rest % ctiles);
        g = rest / ctiles;
    } else {
        ct = int(bid % ctiles);
        const int64_t rest = bid / ctiles;
        mt = int(rest % mtiles);
        g = rest / mtiles;
    }
    const int64_t i0 = d.gfirst[g];
    const int64_t icount = d.gfirst[g + 1] - i0;
    const int N = 1 << d.nb;
    const int64_t M = int64_t(1) << d.mb;
    const int K = 1 << d.kb;
    const int64_t cols = icount * N;
    const int64_t c0 = int64_t(ct) * GBN;
    if (c0 >= cols) return;  // uniform across the block
    const int64_t m0 = int64_t(mt) * GBM;
    if (tid < 40) {
        s_pAm[tid] = d.pAm[tid];
        s_pCm[tid] = d.pCm[tid];
    }
    if (tid == 0) {
        const int64_t sig = i0 / d.nOut, beta = i0 - sig * d.nOut;
        s_ia = int64_t(d.sigA[sig]) * d.nOutA + d.outA[beta];
        s_ea = d.mxA ? exp_of(d.mxA[s_ia]) : 0;
    }
    __syncthreads();
    if (tid < GBM) {
        const int64_t m = m0 + tid;
        s_offA[tid] = m < M ? dep(m, s_pAm, d.mb) : 0;
        s_offC[tid] = m < M ? dep(m, s_pCm, d.mb) : 0;
    } else if (tid < GBM + GBN) {
        const int c = tid - GBM;
        const int64_t gc = c0 + c;
        s_mx[c] = 0;
        if (gc < cols) {
            const int64_t inst = i0 + gc / N;
            const int n = int(gc % N);
            const int64_t sig = inst / d.nOut, beta = inst - sig * d.nOut;
            const int64_t ib = int64_t(d.sigB[sig]) * d.nOutB + d.outB[beta];
            s_bbase[c] = ib * d.sB + dep(n, d.pBn, d.nb);
            s_cbase[c] = inst * d.sC + dep(n, d.pCn, d.nb);
            const int eb = d.mxB ? exp_of(d.mxB[ib]) : 0;
            s_eb[c] = eb;
            if (n == 0 && mt == 0) d.EC[inst] = d.EA[s_ia] + s_ea + d.EB[ib] + eb;
        } else {
            s_bbase[c] = -1;
            s_cbase[c] = -1;
            s_eb[c] = 0;
        }
    }
    __syncthreads();
    const float2 *A = d.A + s_ia * d.sA;
    const int tm = tid & 15, tn = tid >> 4;
    float2 acc[8][4];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = make_float2(0.f, 0.f);
    const int bk = K < GBK ? K : GBK;
    for (int k0 = 0; k0 < K; k0 += bk) {
        for (int e = tid; e < bk * GBM; e += 256) {
            const int kk = e % bk, r = e / bk;
            float2 v = make_float2(0.f, 0.f);
            if (m0 + r < M) v = __ldg(A + s_offA[r] + k0 + kk);
            s_A[kk][r] = v;
        }
        for (int e = tid; e < bk * GBN; e += 256) {
            const int kk = e % bk, c = e / bk;
            float2 v = make_float2(0.f, 0.f);
            if (s_bbase[c] >= 0) v = __ldg(d.B + s_bbase[c] + k0 + kk);
            s_B[kk][c] = v;
        }
        __syncthreads();
        for (int kk = 0; kk < bk; ++kk) {
            float2 a[8], b[4];
#pragma unroll
            for (int x = 0; x < 8; ++x) a[x] = s_A[kk][tm + 16 * x];
#pragma unroll
            for (int y = 0; y < 4; ++y) b[y] = s_B[kk][4 * tn + y];
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) cfma(acc[x][y], a[x], b[y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int c = 4 * tn + y;
        if (s_cbase[c] < 0) continue;
        const float sc = pow2f(-(s_ea + s_eb[c]));
        uint32_t mx = 0;
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int r = tm + 16 * x;
            if (m0 + r >= M) continue;
            const float2 v = make_float2(acc[x][y].x * sc, acc[x][y].y * sc);
            d.C[s_cbase[c] + s_offC[r]] = v;
            mx = max(mx, absmax_bits(v));
        }
        if (d.mxC) {  // lanes tn*16 .. tn*16+15 share column c: reduce each half-warp first
            const unsigned half = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
            const uint32_t r = __reduce_max_sync(half, mx);
            if (tm == 0 && r) atomicMax(&s_mx[c], r);
        }
    }
    if (d.mxC) {
        __syncthreads();
        if (tid < GBN && s_cbase[tid] >= 0) {
            const int64_t inst = i0 + (c0 + tid) / N;
            record_max(d.mxC + inst, s_mx[tid]);
        }
    }
}

// Grouped SIMT complex GEMM, FP32 FMA, K >= 2: the same 128 x 64 tiles
// and block order as k_step_gemm_simt, 128 threads of 8 x 8 complex
// outputs each (rows tm + 16 x, columns 8 tn + y), K in chunks of up to 16
// staged in shared memory by cp.async in two stages, so that a chunk's
// loads run while the previous chunk is multiplied.  Shared memory holds A
// and B K-contiguous per row / column (the operands' own order), rows
// padded to 18 complex (144 bytes) so that the 16-byte reads of eight lanes
// on consecutive rows touch every bank once.
constexpr int SBM = 128, SBN = 64, SBK = 16, SLD = 18;
constexpr size_t SIMT2_SMEM = size_t(2) * (SBM + SBN) * SLD * sizeof(float2);

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

__global__ void __launch_bounds__(128) k_step_gemm_simt2(const StepDesc d, int ctiles, int mtiles) {
    extern __shared__ __align__(16) float2 s2[];
    __shared__ int64_t s_offC[SBM];
    __shared__ int64_t s_bbase[SBN], s_cbase[SBN];
    __shared__ int32_t s_eb[SBN];
    __shared__ uint32_t s_mx[SBN];
    __shared__ int64_t s_ia;
    __shared__ int s_ea;
    const int tid = threadIdx.x;
    const int64_t bid = blockIdx.x;
    int mt, ct;
    int64_t g;
    if (d.sched == 0) {
        mt = int(bid % mtiles);
        const int64_t rest = bid / mtiles;
        ct = int(rest % ctiles);
        g = rest / ctiles;
    } else {
        ct = int(bid % ctiles);
        const int64_t rest = bid / ctiles;
        mt = int(rest % mtiles);
        g = rest / mtiles;
    }
    const int64_t i0 = d.gfirst[g];
    const int64_t icount = d.gfirst[g + 1] - i0;
    const int N = 1 << d.nb;
    const int64_t M = int64_t(1) << d.mb;
    const int K = 1 << d.kb;
    const int64_t cols = icount * N;
    const int64_t c0 = int64_t(ct) * SBN;
    if (c0 >= cols) return;  // uniform across the block
    const int64_t m0 = int64_t(mt) * SBM;
    if (tid == 0) {
        const int64_t sig = i0 / d.nOut, beta = i0 - sig * d.nOut;
        s_ia = int64_t(d.sigA[sig]) * d.nOutA + d.outA[beta];
        s_ea = d.mxA ? exp_of(d.mxA[s_ia]) : 0;
    }
    __syncthreads();
    {
        const int64_t m = m0 + tid;
        s_offC[tid] = m < M ? dep(m, d.pCm, d.mb) : 0;
    }
    if (tid < SBN) {
        const int c = tid;
        const int64_t gc = c0 + c;
        s_mx[c] = 0;
        if (gc < cols) {
            const int64_t inst = i0 + gc / N;
            const int n = int(gc % N);
            const int64_t sig = inst / d.nOut, beta = inst - sig * d.nOut;
            const int64_t ib = int64_t(d.sigB[sig]) * d.nOutB + d.outB[beta];
            s_bbase[c] = ib * d.sB + (int64_t(n) << d.kb);  // B is K-major and affine
            s_cbase[c] = inst * d.sC + dep(n, d.pCn, d.nb);
            const int eb = d.mxB ? exp_of(d.mxB[ib]) : 0;
            s_eb[c] = eb;
            if (n == 0 && mt == 0) d.EC[inst] = d.EA[s_ia] + s_ea + d.EB[ib] + eb;
        } else {
            s_bbase[c] = -1;
            s_cbase[c] = -1;
            s_eb[c] = 0;
        }
    }
    __syncthreads();
    const float2 *A = d.A + s_ia * d.sA;  // row m at m * K: K-major and affine
    const int bk = K < SBK ? K : SBK;      // complex k per chunk (even: K >= 2)
    const int pieces = bk >> 1;            // 16-byte pieces per row / column and chunk
    const int nchunk = K / bk;
    // stage st: A at s2 + st * SBM * SLD, B at s2 + 2 * SBM * SLD + st * SBN * SLD
    // one chunk's cp.async: piece q of row r at (r, 2q); consecutive threads
    // take consecutive pieces of a row (coalesced)
    auto issue = [&](int ch, int st) {
        const int k0 = ch * bk;
        for (int e = tid; e < SBM * pieces; e += 128) {
            const int r = e / pieces, q = e - r * pieces;
            const bool v = m0 + r < M;
            const float2 *src = v ? A + ((m0 + r) << d.kb) + k0 + 2 * q : A;
            cp_async16_zfill(static_cast<uint32_t>(__cvta_generic_to_shared(s2 + st * SBM * SLD + r * SLD + 2 * q)), src,
                             v);
        }
        for (int e = tid; e < SBN * pieces; e += 128) {
            const int c = e / pieces, q = e - c * pieces;
            const int64_t bb = s_bbase[c];
            const bool v = bb >= 0;
            const float2 *src = v ? d.B + bb + k0 + 2 * q : d.B;
            cp_async16_zfill(
                static_cast<uint32_t>(__cvta_generic_to_shared(s2 + 2 * SBM * SLD + st * SBN * SLD + c * SLD + 2 * q)),
                src, v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int tm = tid & 15, tn = tid >> 4;
    float2 acc[8][8];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = make_float2(0.f, 0.f);
    issue(0, 0);
    for (int ch = 0; ch < nchunk; ++ch) {
        if (ch + 1 < nchunk) {
            issue(ch + 1, (ch + 1) & 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float2 *a_s = s2 + (ch & 1) * SBM * SLD + tm * SLD;
        const float2 *b_s = s2 + 2 * SBM * SLD + (ch & 1) * SBN * SLD + (8 * tn) * SLD;
        for (int kk = 0; kk < bk; kk += 2) {
            float4 a[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) a[x] = *reinterpret_cast<const float4 *>(a_s + 16 * x * SLD + kk);
#pragma unroll
            for (int y = 0; y < 8; ++y) {
                const float4 b = *reinterpret_cast<const float4 *>(b_s + y * SLD + kk);
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    cfma(acc[x][y], make_float2(a[x].x, a[x].y), make_float2(b.x, b.y));
                    cfma(acc[x][y], make_float2(a[x].z, a[x].w), make_float2(b.z, b.w));
                }
            }
        }
        __syncthreads();  // the stage is refilled two chunks later
    }
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int c = 8 * tn + y;
        if (s_cbase[c] < 0) continue;
        const float sc = pow2f(-(s_ea + s_eb[c]));
        uint32_t mx = 0;
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int r = tm + 16 * x;
            if (m0 + r >= M) continue;
            const float2 v = make_float2(acc[x][y].x * sc, acc[x][y].y * sc);
            d.C[s_cbase[c] + s_offC[r]] = v;
            mx = max(mx, absmax_bits(v));
        }
        if (d.mxC) {  // lanes tn*16 .. tn*16+15 share column c: reduce each half-warp first
            const unsigned half = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
            const uint32_t r = __reduce_max_sync(half, mx);
            if (tm == 0 && r) atomicMax(&s_mx[c], r);
        }
    }
    if (d.mxC) {
        __syncthreads();
        if (tid < SBN && s_cbase[tid] >= 0) {
            const int64_t inst = i0 + (c0 + tid) / N;
            record_max(d.mxC + inst, s_mx[tid]);
        }
    }
}

// Steps with at most four outputs per instance (M N <= 4) and a long K:
// each output C[i](m, n) = sum_k A[a(i)](m, k) B[b(i)](k, n) is one dot
// product of two K-contiguous complex runs, computed by one block (16-byte
// loads, FP32 FMA, a fixed-order block reduction), scaled by the operands'
// power-of-two factors and stored with its instance's exponent and max.
__global__ void __launch_bounds__(256) k_step_dot(const StepDesc d) {
    __shared__ float2 s_part[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mn_log = d.mb + d.nb;
    const int64_t i = int64_t(blockIdx.x) >> mn_log;
    const int mn = int(blockIdx.x & ((1u << mn_log) - 1));
    const int m = mn >> d.nb, n = mn & ((1 << d.nb) - 1);
    const int2 ab = d.instab[i];
    const int K = 1 << d.kb;
    const float4 *a4 = reinterpret_cast<const float4 *>(d.A + int64_t(ab.x) * d.sA + (int64_t(m) << d.kb));
    const float4 *b4 = reinterpret_cast<const float4 *>(d.B + int64_t(ab.y) * d.sB + (int64_t(n) << d.kb));
    float2 acc = make_float2(0.f, 0.f), acc2 = make_float2(0.f, 0.f);
    for (int q = tid; q < K / 2; q += 256) {
        const float4 x = __ldg(a4 + q), y = __ldg(b4 + q);
        cfma(acc, make_float2(x.x, x.y), make_float2(y.x, y.y));
        cfma(acc2, make_float2(x.z, x.w), make_float2(y.z, y.w));
    }
    acc.x += acc2.x;
    acc.y += acc2.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) s_part[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        float2 t = s_part[0];
        for (int w = 1; w < 8; ++w) {
            t.x += s_part[w].x;
            t.y += s_part[w].y;
        }
        const int ea = d.mxA ? exp_of(d.mxA[ab.x]) : 0;
        const int eb = d.mxB ? exp_of(d.mxB[ab.y]) : 0;
        const float sc = pow2f(-(ea + eb));
        const float2 v = make_float2(t.x * sc, t.y * sc);
        d.C[i * d.sC + dep(m, d.pCm, d.mb) + dep(n, d.pCn, d.nb)] = v;
        if (mn == 0) d.EC[i] = d.EA[ab.x] + ea + d.EB[ab.y] + eb;
        const uint32_t mx = absmax_bits(v);
        if (d.mxC && mx) record_max(d.mxC + i, mx);
    }
}

// root entry of completion x: its r bits reversed (root bit t = the t-th
// lowest open qubit; x's most significant bit = the lowest open qubit)
__device__ __forceinline__ int64_t root_entry(int64_t x, int r) {
    return r == 0 ? 0 : int64_t(__brevll(uint64_t(x)) >> (64 - r));
}

// one thread per (input row, completion): amps[p 2^r + x] += the sum over
// the pass's slice instances, in slice order, of root entry x times 2^E
__global__ void k_accumulate(const float2 *__restrict__ root, const int32_t *__restrict__ E,
                             const int32_t *__restrict__ uniq, int64_t k, int64_t n_sig, int32_t n_out, int r,
                             double2 *__restrict__ amps) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= (k << r)) return;
    const int64_t p = q >> r, x = q & ((int64_t(1) << r) - 1);
    const int64_t beta = uniq[p], j = root_entry(x, r);
    double re = 0.0, im = 0.0;
    for (int64_t s = 0; s < n_sig; ++s) {
        const int64_t idx = s * n_out + beta;
        const float2 v = root[(idx << r) + j];
        const int e = E[idx];
        re += ldexp(double(v.x), e);
        im += ldexp(double(v.y), e);
    }
    double2 a = amps[q];
    a.x += re;
    a.y += im;
    amps[q] = a;
}

__global__ void k_extract(const float2 *__restrict__ root, const int32_t *__restrict__ E,
                          const int32_t *__restrict__ uniq, int64_t k, int64_t sigma, int32_t n_out, int r,
                          double2 *__restrict__ out) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= (k << r)) return;
    const int64_t p = q >> r, x = q & ((int64_t(1) << r) - 1);
    const int64_t idx = sigma * n_out + uniq[p];
    const float2 v = root[(idx << r) + root_entry(x, r)];
    out[q] = make_double2(ldexp(double(v.x), E[idx]), ldexp(double(v.y), E[idx]));
}

__global__ void __launch_bounds__(1024) k_xeb(const double2 *__restrict__ amps, int64_t k, double scale,
                                              double *__restrict__ out) {
    __shared__ double s[1024];
    double acc = 0.0;
    for (int64_t p = threadIdx.x; p < k; p += 1024) {
        const double2 a = amps[p];
        acc += a.x * a.x + a.y * a.y;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = scale * s[0] - 1.0;
}

// x = N |a|^2 in FP64 with explicit round-to-nearest operations (no
// contraction into an FMA), so that a host computing re*re + im*im, then
// times N, gets the same bits
__device__ __forceinline__ double pt_x(double2 a, double n_states) {
    return __dmul_rn(n_states, __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)));
}

// Sums over the k amplitudes, for the mixture density
// p(x) = e^-x (1 + F (x - 1)) of x = N |amp|^2 (fidelity F; Eq. fxeb):
// out[0] = sum g, out[1] = sum g^2 with g = (x - 1) / (1 + F (x - 1)) (the
// log-likelihood's first derivative and minus its second), out[2] = sum
// log(1 + F (x - 1)), out[3] = sum x, out[4] = sum x^2.  One block, fixed
// order.
__global__ void __launch_bounds__(1024) k_pt_moments(const double2 *__restrict__ amps, int64_t k, double n_states,
                                                     double fid, double *__restrict__ out) {
    __shared__ double s[5][1024];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
    for (int64_t p = threadIdx.x; p < k; p += 1024) {
        const double x = pt_x(amps[p], n_states);
        const double d = 1.0 + fid * (x - 1.0);
        const double g = (x - 1.0) / d;
        a0 += g;
        a1 += g * g;
        a2 += log(d);
        a3 += x;
        a4 += x * x;
    }
    s[0][threadIdx.x] = a0;
    s[1][threadIdx.x] = a1;
    s[2][threadIdx.x] = a2;
    s[3][threadIdx.x] = a3;
    s[4][threadIdx.x] = a4;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 5; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = s[threadIdx.x][0];
}

// counts[j] += #{b : j width <= x_b < (j + 1) width}, j < nbins, with
// width = x_max / nbins; counts[nbins] gathers x_b >= x_max.  The bin is
// floor(x / width) in FP64 (correctly rounded division), integer atomics.
__global__ void k_pt_hist(const double2 *__restrict__ amps, int64_t k, double n_states, double x_max, int nbins,
                          unsigned long long *__restrict__ counts) {
    extern __shared__ unsigned int h[];  // nbins + 1 block-local counts
    for (int j = threadIdx.x; j <= nbins; j += blockDim.x) h[j] = 0u;
    __syncthreads();
    const double width = __ddiv_rn(x_max, double(nbins));
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < k; p += int64_t(gridDim.x) * blockDim.x) {
        const double q = floor(__ddiv_rn(pt_x(amps[p], n_states), width));
        const int j = q < double(nbins) ? int(q) : nbins;
        atomicAdd(&h[j], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= nbins; j += blockDim.x)
        if (h[j]) atomicAdd(&counts[j], (unsigned long long)h[j]);
}

// Row p's batch a[p 2^r .. p 2^r + 2^r): with u = uniform[p] in [0, 1), the
// smallest x whose running sum of |a_x|^2 exceeds u times the batch total
// (2^r - 1 if none does); FP64, correctly rounded operations in x order.
__global__ void k_sample(const double2 *__restrict__ amps, int64_t k, int r, const double *__restrict__ uniform,
                         int64_t *__restrict__ picks) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= k) return;
    const double2 *a = amps + (p << r);
    const int64_t n = int64_t(1) << r;
    double tot = 0.0;
    for (int64_t x = 0; x < n; ++x) {
        const double2 v = a[x];
        tot = __dadd_rn(tot, __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)));
    }
    const double thr = __dmul_rn(uniform[p], tot);
    double c = 0.0;
    int64_t pick = n - 1;
    for (int64_t x = 0; x < n; ++x) {
        const double2 v = a[x];
        c = __dadd_rn(c, __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)));
        if (c > thr) {
            pick = x;
            break;
        }
    }
    picks[p] = pick;
}

// FP32 fused multiply-add throughput probe: each thread runs 8 independent
// FMA chains for `iters` rounds (16 flops per round); the result is stored
// only under a condition the values never meet, so the work is kept.
__global__ void __launch_bounds__(256) k_fma_probe(int64_t iters, float seed, float *out) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + float(threadIdx.x + j);
    const float b = 0.999999f, c = 1e-6f;
#pragma unroll 4
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == -1.f) out[blockIdx.x] = s;
}

}  // namespace

cudaError_t launch_fill(const FillJobD *jobs, int64_t njobs, const LeafHighD *highs, int64_t batch, float2 *ws,
                        cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    const int64_t threads = njobs * 32;
    const int64_t blocks = (threads + 255) / 256;
    k_fill<<<dim3((unsigned)blocks), 256, 0, s>>>(jobs, njobs, highs, batch, ws);
    return cudaGetLastError();
}

// Lanes per row of the row kernel: as few as keep a lane's share of the
// row's K * N products within 64 (fewer cross-lane sums per output), at
// least K / 32 (a lane holds at most 32 complex A values) and at most 8
// (and K / 2: a lane loads 16 bytes at a time).
static int row_lanes(int kb, int nb) {
    const int K = 1 << kb;
    int L = (K << nb) >> 6;
    L = L < 1 ? 1 : (L > 8 ? 8 : L);
    if (L < K / 32) L = K / 32;
    if (K >= 2 && L > K / 2) L = K / 2;
    return L;
}

cudaError_t launch_step_row(const StepDesc &d, cudaStream_t s) {
    if (d.kb + d.nb > 8 || d.nb > 4 || d.mb > 40) return cudaErrorInvalidValue;
    const int K = 1 << d.kb;
    const int L = row_lanes(d.kb, d.nb);
    const int R = 32 / L;
    const int KL = K / L;
    if ((d.nb == 4 && KL > 4) || (d.nb == 3 && KL > 8) || (d.nb == 2 && KL > 16) || KL > 32)
        return cudaErrorInvalidValue;  // no instance of the kernel for this split
    const int64_t M = int64_t(1) << d.mb;
    int64_t blocks, mblocks = 1;
    int rows_per_block;
    if (M >= 8 * R) {  // blocks inside one group: up to 16 (schedule 1: 4) passes of 8 warps x R rows
        int64_t passes = M / (8 * R);
        const int64_t cap = d.sched == 0 ? 16 : 4;
        passes = passes > cap ? cap : passes;
        rows_per_block = int(8 * R * passes);
        mblocks = M / rows_per_block;
        blocks = d.n_groups * mblocks;
    } else {  // small instances: 4 passes over consecutive (group, row) / schedule 1: (instance, row) pairs
        rows_per_block = 8 * R * 4;
        blocks = (((d.sched == 1 ? d.nInst : d.n_groups) << d.mb) + rows_per_block - 1) / rows_per_block;
    }
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const dim3 g((unsigned)blocks);
#define TN_ROW(NB_, KL_) k_step_row<NB_, KL_><<<g, ROW_THREADS, 0, s>>>(d, rows_per_block, mblocks)
    // KL = K / L for K * N <= 256: NB 0-1 up to 32, NB 2 up to 16, NB 3 up
    // to 8, NB 4 up to 4 (row_lanes keeps 2 KL + 2 N <= 72 registers)
#define TN_ROW_KL(NB_)                                         \
    switch (KL) {                                              \
        case 1: TN_ROW(NB_, 1); break;                         \
        case 2: TN_ROW(NB_, 2); break;                         \
        case 4: TN_ROW(NB_, 4); break;                         \
        case 8: TN_ROW(NB_, (NB_ <= 3 ? 8 : 4)); break;        \
        case 16: TN_ROW(NB_, (NB_ <= 2 ? 16 : 4)); break;      \
        default: TN_ROW(NB_, (NB_ <= 1 ? 32 : 4)); break;      \
    }
    switch (d.nb) {
        case 0: TN_ROW_KL(0); break;
        case 1: TN_ROW_KL(1); break;
        case 2: TN_ROW_KL(2); break;
        case 3: TN_ROW_KL(3); break;
        default: TN_ROW_KL(4); break;
    }
#undef TN_ROW_KL
#undef TN_ROW
    return cudaGetLastError();
}

cudaError_t launch_step_gemm_simt(const StepDesc &d, cudaStream_t s) {
    const int64_t M = int64_t(1) << d.mb;
    const int64_t N = int64_t(1) << d.nb;
    const int64_t ctiles = (int64_t(d.max_group) * N + GBN - 1) / GBN;
    const int64_t mtiles = (M + GBM - 1) / GBM;
    const int64_t blocks = d.n_groups * ctiles * mtiles;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL || ctiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    static_assert(SBM == GBM && SBN == GBN, "both SIMT GEMMs tile alike");
    if (d.kb >= 1) {  // K >= 2: 16-byte pieces of A rows and B columns
        k_step_gemm_simt2<<<dim3((unsigned)blocks), 128, SIMT2_SMEM, s>>>(d, (int)ctiles, (int)mtiles);
    } else {
        k_step_gemm_simt<<<dim3((unsigned)blocks), 256, 0, s>>>(d, (int)ctiles, (int)mtiles);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_dot(const StepDesc &d, cudaStream_t s) {
    if (d.mb + d.nb > 2 || d.kb < 6) return cudaErrorInvalidValue;
    const int64_t blocks = d.nInst << (d.mb + d.nb);
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_step_dot<<<dim3((unsigned)blocks), 256, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t init_simt_kernels() {
    return cudaFuncSetAttribute(k_step_gemm_simt2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SIMT2_SMEM));
}

cudaError_t launch_accumulate(const float2 *root, const int32_t *E, const int32_t *uniq, int64_t k,
                              int64_t n_sig, int32_t n_out, int r, double *amps, cudaStream_t s) {
    if (k == 0) return cudaSuccess;
    if (r < 0 || r > 30) return cudaErrorInvalidValue;
    const int64_t blocks = ((k << r) + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_accumulate<<<dim3((unsigned)blocks), 256, 0, s>>>(root, E, uniq, k, n_sig, n_out, r,
                                                        reinterpret_cast<double2 *>(amps));
    return cudaGetLastError();
}

cudaError_t launch_extract(const float2 *root, const int32_t *E, const int32_t *uniq, int64_t k, int64_t sigma,
                           int32_t n_out, int r, double *out, cudaStream_t s) {
    if (k == 0) return cudaSuccess;
    if (r < 0 || r > 30) return cudaErrorInvalidValue;
    const int64_t blocks = ((k << r) + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_extract<<<dim3((unsigned)blocks), 256, 0, s>>>(root, E, uniq, k, sigma, n_out, r,
                                                     reinterpret_cast<double2 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_xeb(const double *amps, int64_t k, double scale, double *out, cudaStream_t s) {
    k_xeb<<<1, 1024, 0, s>>>(reinterpret_cast<const double2 *>(amps), k, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_sample(const double *amps, int64_t k, int r, const double *uniform, int64_t *picks,
                          cudaStream_t s) {
    if (k == 0) return cudaSuccess;
    k_sample<<<dim3((unsigned)((k + 127) / 128)), 128, 0, s>>>(reinterpret_cast<const double2 *>(amps), k, r,
                                                               uniform, picks);
    return cudaGetLastError();
}

cudaError_t launch_pt_moments(const double *amps, int64_t k, double n_states, double fid, double *out,
                              cudaStream_t s) {
    k_pt_moments<<<1, 1024, 0, s>>>(reinterpret_cast<const double2 *>(amps), k, n_states, fid, out);
    return cudaGetLastError();
}

cudaError_t launch_pt_hist(const double *amps, int64_t k, double n_states, double x_max, int nbins,
                           unsigned long long *counts, cudaStream_t s) {
    const int64_t want = (k + 255) / 256;
    const int blocks = int(want < 1024 ? (want > 0 ? want : 1) : 1024);
    k_pt_hist<<<blocks, 256, size_t(nbins + 1) * sizeof(unsigned int), s>>>(reinterpret_cast<const double2 *>(amps),
                                                                         k, n_states, x_max, nbins, counts);
    return cudaGetLastError();
}

cudaError_t launch_fma_probe(int64_t blocks, int64_t iters, float *out, cudaStream_t s) {
    if (blocks <= 0 || blocks > 0x7fffffffLL || iters < 0) return cudaErrorInvalidValue;
    k_fma_probe<<<dim3((unsigned)blocks), 256, 0, s>>>(iters, 1.0f, out);
    return cudaGetLastError();
}

}  // namespace tnk
