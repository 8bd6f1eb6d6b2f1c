// CUDA-core kernels of the contraction path (sm_103a).
//
//   k_fill           leaf instance blocks for one slice batch (the fused gate
//                    tensors with output legs projected on the bitstrings'
//                    values and sliced legs on the slice's values)
//   k_step_row       one pairwise step C = A (x) B with a small B operand
//                    (K*N <= 64): one thread per row m of A, the B block of the
//                    instance in shared memory; the bandwidth-bound
//                    "high-rank x low-rank" contraction of SM Sec. V.A
//   k_step_gemm_simt tiled complex GEMM with gathered (bit-permuted) operand
//                    loads, FP32 FMA; the plain FP32 form of big x big steps
//   k_accumulate     amp[p] += sum over the batch's slices of the root
//                    partials times 2^E, complex128, fixed slice order
//                    (first-level slicing, SM Sec. IV.B)
//   k_xeb            FP64 fixed-order reduction of sum |amp|^2 (Eq. fxeb)
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
__device__ __forceinline__ void record_max(uint32_t *slot, uint32_t v) {
    if (v > __ldcg(slot)) atomicMax(slot, v);
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

// K*N <= 64; NB = log2 N (0..4).
template <int NB>
__global__ void __launch_bounds__(ROW_THREADS) k_step_row(const StepDesc d) {
    constexpr int N = 1 << NB;
    __shared__ int8_t s_pos[4][40];
    __shared__ int64_t s_offAk[64];
    __shared__ int64_t s_offB[64];
    __shared__ int64_t s_mlo[ROW_THREADS];
    __shared__ float2 s_B[64];
    __shared__ int64_t s_hi;
    __shared__ int64_t s_ia, s_ib;
    __shared__ float s_sa;
    const int tid = threadIdx.x;
    const int K = 1 << d.kb;
    const int mb = d.mb;
    const int64_t M = int64_t(1) << mb;
    if (tid < 40) {
        s_pos[0][tid] = d.pAm[tid];
        s_pos[1][tid] = tid < 24 ? d.pAk[tid] : 0;
        s_pos[2][tid] = tid < 24 ? d.pBk[tid] : 0;
        s_pos[3][tid] = tid < 24 ? d.pBn[tid] : 0;
    }
    __syncthreads();
    if (tid < K) s_offAk[tid] = dep(tid, s_pos[1], d.kb);
    if (tid < K * N) {
        const int k = tid >> NB, n = tid & (N - 1);
        s_offB[tid] = dep(k, s_pos[2], d.kb) + dep(n, s_pos[3], NB);
    }
    const int lob = mb < 8 ? mb : 8;
    s_mlo[tid] = dep(tid & ((1 << lob) - 1), s_pos[0], lob);
    const int64_t gid0 = int64_t(blockIdx.x) * ROW_THREADS;
    const bool uniform = M >= ROW_THREADS;  // whole block inside one instance
    if (uniform && tid == 0 && gid0 < (d.nInst << mb)) {
        const int64_t i = gid0 >> mb;
        const int64_t sig = i / d.nOut, beta = i - sig * d.nOut;
        s_ia = int64_t(d.sigA[sig]) * d.nOutA + d.outA[beta];
        s_ib = int64_t(d.sigB[sig]) * d.nOutB + d.outB[beta];
        s_hi = mb > 8 ? dep((gid0 & (M - 1)) >> 8, s_pos[0] + 8, mb - 8) : 0;
    }
    __syncthreads();
    if (uniform && gid0 < (d.nInst << mb)) {
        if (tid < K * N) {
            const float sb = pow2f(-(d.mxB ? exp_of(d.mxB[s_ib]) : 0));
            const float2 b = d.B[s_ib * d.sB + s_offB[tid]];
            s_B[tid] = make_float2(b.x * sb, b.y * sb);
        }
        if (tid == 0) s_sa = pow2f(-(d.mxA ? exp_of(d.mxA[s_ia]) : 0));
        __syncthreads();
    }
    const int64_t gid = gid0 + tid;
    if (gid >= (d.nInst << mb)) return;
    const int64_t i = gid >> mb;
    const int64_t m = gid & (M - 1);
    int64_t ia, ib, offm;
    float sa;
    int ea = 0, eb = 0;
    if (uniform) {
        ia = s_ia;
        ib = s_ib;
        offm = s_hi + s_mlo[tid];
        sa = s_sa;
    } else {
        const int64_t sig = i / d.nOut, beta = i - sig * d.nOut;
        ia = int64_t(d.sigA[sig]) * d.nOutA + d.outA[beta];
        ib = int64_t(d.sigB[sig]) * d.nOutB + d.outB[beta];
        offm = s_mlo[m & 255];
        ea = d.mxA ? exp_of(d.mxA[ia]) : 0;
        sa = pow2f(-ea);
    }
    const float2 *A = d.A + ia * d.sA + offm;
    float2 acc[N];
#pragma unroll
    for (int n = 0; n < N; ++n) acc[n] = make_float2(0.f, 0.f);
    if (uniform) {
        for (int k = 0; k < K; ++k) {
            float2 a = __ldg(A + s_offAk[k]);
            a.x *= sa;
            a.y *= sa;
#pragma unroll
            for (int n = 0; n < N; ++n) cfma(acc[n], a, s_B[k * N + n]);
        }
    } else {
        eb = d.mxB ? exp_of(d.mxB[ib]) : 0;
        const float sb = pow2f(-eb);
        const float2 *B = d.B + ib * d.sB;
        for (int k = 0; k < K; ++k) {
            float2 a = __ldg(A + s_offAk[k]);
            a.x *= sa;
            a.y *= sa;
#pragma unroll
            for (int n = 0; n < N; ++n) {
                float2 b = __ldg(B + s_offB[k * N + n]);
                b.x *= sb;
                b.y *= sb;
                cfma(acc[n], a, b);
            }
        }
    }
    float2 *C = d.C + i * d.sC + m * N;
    uint32_t mx = 0;
    if constexpr (N >= 2) {
#pragma unroll
        for (int n = 0; n < N; n += 2) {
            reinterpret_cast<float4 *>(C)[n / 2] = make_float4(acc[n].x, acc[n].y, acc[n + 1].x, acc[n + 1].y);
            mx = max(mx, max(absmax_bits(acc[n]), absmax_bits(acc[n + 1])));
        }
    } else {
        C[0] = acc[0];
        mx = absmax_bits(acc[0]);
    }
    if (m == 0) {
        if (uniform) {
            ea = d.mxA ? exp_of(d.mxA[ia]) : 0;
            eb = d.mxB ? exp_of(d.mxB[ib]) : 0;
        }
        d.EC[i] = d.EA[ia] + ea + d.EB[ib] + eb;
    }
    if (d.mxC) {
        if (M >= 32) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if ((tid & 31) == 0) record_max(d.mxC + i, mx);
        } else {
            record_max(d.mxC + i, mx);
        }
    }
}

// Tiled FP32 complex GEMM with gathered operands: tile 64 (m) x 32 (n) x 8 (k),
// 256 threads, 4 x 2 outputs per thread.
constexpr int GBM = 64, GBN = 32, GBK = 8;

__global__ void __launch_bounds__(256) k_step_gemm_simt(const StepDesc d) {
    __shared__ int8_t s_pos[4][40];
    __shared__ int64_t s_offAm[GBM];
    __shared__ int64_t s_offBn[GBN];
    __shared__ float2 s_A[GBK][GBM + 1];
    __shared__ float2 s_B[GBK][GBN + 1];
    __shared__ int64_t s_ia, s_ib;
    __shared__ float s_sa, s_sb;
    __shared__ int s_ea, s_eb;
    const int tid = threadIdx.x;
    const int64_t M = int64_t(1) << d.mb;
    const int N = 1 << d.nb;
    const int64_t K = int64_t(1) << d.kb;
    const int64_t tiles_m = (M + GBM - 1) / GBM;
    const int64_t tiles_n = (N + GBN - 1) / GBN;
    const int64_t per_inst = tiles_m * tiles_n;
    const int64_t t = blockIdx.x;
    const int64_t i = t / per_inst;
    const int64_t r = t - i * per_inst;
    const int64_t m0 = (r / tiles_n) * GBM;
    const int64_t n0 = (r % tiles_n) * GBN;
    if (tid < 40) {
        s_pos[0][tid] = d.pAm[tid];
        s_pos[1][tid] = tid < 24 ? d.pAk[tid] : 0;
        s_pos[2][tid] = tid < 24 ? d.pBk[tid] : 0;
        s_pos[3][tid] = tid < 24 ? d.pBn[tid] : 0;
    }
    if (tid == 0) {
        const int64_t sig = i / d.nOut, beta = i - sig * d.nOut;
        s_ia = int64_t(d.sigA[sig]) * d.nOutA + d.outA[beta];
        s_ib = int64_t(d.sigB[sig]) * d.nOutB + d.outB[beta];
        s_ea = d.mxA ? exp_of(d.mxA[s_ia]) : 0;
        s_eb = d.mxB ? exp_of(d.mxB[s_ib]) : 0;
        s_sa = pow2f(-s_ea);
        s_sb = pow2f(-s_eb);
    }
    __syncthreads();
    if (tid < GBM) s_offAm[tid] = (m0 + tid < M) ? dep(m0 + tid, s_pos[0], d.mb) : 0;
    else if (tid < GBM + GBN) {
        const int c = tid - GBM;
        s_offBn[c] = (n0 + c < N) ? dep(n0 + c, s_pos[3], d.nb) : 0;
    }
    __syncthreads();
    const float2 *A = d.A + s_ia * d.sA;
    const float2 *B = d.B + s_ib * d.sB;
    const float sa = s_sa, sb = s_sb;
    const int tm = (tid % 16) * 4;  // 4 rows
    const int tn = (tid / 16) * 2;  // 2 cols
    float2 acc[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 2; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < K; k0 += GBK) {
        // A tile: 8 x 64 entries, 2 per thread
        for (int e = tid; e < GBK * GBM; e += 256) {
            const int kk = e / GBM, mm = e % GBM;
            float2 v = make_float2(0.f, 0.f);
            if (k0 + kk < K && m0 + mm < M) {
                v = __ldg(A + s_offAm[mm] + dep(k0 + kk, s_pos[1], d.kb));
                v.x *= sa;
                v.y *= sa;
            }
            s_A[kk][mm] = v;
        }
        for (int e = tid; e < GBK * GBN; e += 256) {
            const int kk = e / GBN, nn = e % GBN;
            float2 v = make_float2(0.f, 0.f);
            if (k0 + kk < K && n0 + nn < N) {
                v = __ldg(B + dep(k0 + kk, s_pos[2], d.kb) + s_offBn[nn]);
                v.x *= sb;
                v.y *= sb;
            }
            s_B[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float2 a[4], b[2];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = s_A[kk][tm + x];
#pragma unroll
            for (int y = 0; y < 2; ++y) b[y] = s_B[kk][tn + y];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 2; ++y) cfma(acc[x][y], a[x], b[y]);
        }
        __syncthreads();
    }
    uint32_t mx = 0;
    float2 *C = d.C + i * d.sC;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const int64_t m = m0 + tm + x, n = n0 + tn + y;
            if (m < M && n < N) {
                C[m * N + n] = acc[x][y];
                mx = max(mx, absmax_bits(acc[x][y]));
            }
        }
    if (m0 == 0 && n0 == 0 && tid == 0) d.EC[i] = d.EA[s_ia] + s_ea + d.EB[s_ib] + s_eb;
    if (d.mxC) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) record_max(d.mxC + i, mx);
    }
}

__global__ void k_accumulate(const float2 *__restrict__ root, const int32_t *__restrict__ E,
                             const int32_t *__restrict__ uniq, int64_t k, int64_t n_sig, int32_t n_out,
                             double2 *__restrict__ amps) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= k) return;
    const int64_t beta = uniq[p];
    double re = 0.0, im = 0.0;
    for (int64_t s = 0; s < n_sig; ++s) {
        const int64_t idx = s * n_out + beta;
        const float2 v = root[idx];
        const int e = E[idx];
        re += ldexp(double(v.x), e);
        im += ldexp(double(v.y), e);
    }
    double2 a = amps[p];
    a.x += re;
    a.y += im;
    amps[p] = a;
}

__global__ void k_extract(const float2 *__restrict__ root, const int32_t *__restrict__ E,
                          const int32_t *__restrict__ uniq, int64_t k, int64_t sigma, int32_t n_out,
                          double2 *__restrict__ out) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= k) return;
    const int64_t idx = sigma * n_out + uniq[p];
    const float2 v = root[idx];
    out[p] = make_double2(ldexp(double(v.x), E[idx]), ldexp(double(v.y), E[idx]));
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

}  // namespace

cudaError_t launch_fill(const FillJobD *jobs, int64_t njobs, const LeafHighD *highs, int64_t batch, float2 *ws,
                        cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    const int64_t threads = njobs * 32;
    const int64_t blocks = (threads + 255) / 256;
    k_fill<<<dim3((unsigned)blocks), 256, 0, s>>>(jobs, njobs, highs, batch, ws);
    return cudaGetLastError();
}

cudaError_t launch_step_row(const StepDesc &d, cudaStream_t s) {
    if (d.kb + d.nb > 6 || d.nb > 4 || d.mb > 40) return cudaErrorInvalidValue;
    const int64_t rows = d.nInst << d.mb;
    const int64_t blocks = (rows + ROW_THREADS - 1) / ROW_THREADS;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const dim3 g((unsigned)blocks);
    switch (d.nb) {
        case 0: k_step_row<0><<<g, ROW_THREADS, 0, s>>>(d); break;
        case 1: k_step_row<1><<<g, ROW_THREADS, 0, s>>>(d); break;
        case 2: k_step_row<2><<<g, ROW_THREADS, 0, s>>>(d); break;
        case 3: k_step_row<3><<<g, ROW_THREADS, 0, s>>>(d); break;
        default: k_step_row<4><<<g, ROW_THREADS, 0, s>>>(d); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_step_gemm_simt(const StepDesc &d, cudaStream_t s) {
    const int64_t M = int64_t(1) << d.mb;
    const int64_t N = int64_t(1) << d.nb;
    const int64_t tiles = ((M + GBM - 1) / GBM) * ((N + GBN - 1) / GBN) * d.nInst;
    if (tiles <= 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_step_gemm_simt<<<dim3((unsigned)tiles), 256, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const float2 *root, const int32_t *E, const int32_t *uniq, int64_t k,
                              int64_t n_sig, int32_t n_out, double *amps, cudaStream_t s) {
    if (k == 0) return cudaSuccess;
    k_accumulate<<<dim3((unsigned)((k + 255) / 256)), 256, 0, s>>>(root, E, uniq, k, n_sig, n_out,
                                                                   reinterpret_cast<double2 *>(amps));
    return cudaGetLastError();
}

cudaError_t launch_extract(const float2 *root, const int32_t *E, const int32_t *uniq, int64_t k, int64_t sigma,
                           int32_t n_out, double *out, cudaStream_t s) {
    if (k == 0) return cudaSuccess;
    k_extract<<<dim3((unsigned)((k + 255) / 256)), 256, 0, s>>>(root, E, uniq, k, sigma, n_out,
                                                                reinterpret_cast<double2 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_xeb(const double *amps, int64_t k, double scale, double *out, cudaStream_t s) {
    k_xeb<<<1, 1024, 0, s>>>(reinterpret_cast<const double2 *>(amps), k, scale, out);
    return cudaGetLastError();
}

}  // namespace tnk
