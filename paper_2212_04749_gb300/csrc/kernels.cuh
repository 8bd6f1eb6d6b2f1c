// Device-side descriptors and launchers shared by the C ABI (api.cu) and
// the kernels (kernels.cu, gemm_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace tnk {

// One pairwise contraction step, passed by value to every step kernel.
//   C[i](m, n) = sum_k  A[a(i)](m, k) * B[b(i)](k, n)       (complex)
// Instance i = sigma * nOut + beta;  a(i) = sigA[sigma] * nOutA + outA[beta],
// b(i) likewise.  Both operands are K-major and affine: entry (m, k) of an
// A instance sits at element offset k + m * 2^kb (pAm[j] = kb + j), entry
// (k, n) of a B instance at k + n * 2^kb (pBn[j] = kb + j); dep scatters
// the bits of its first argument to the listed bit positions.  C(m, n) of instance i sits at
// i * sC + dep(m, pCm) + dep(n, pCn).  Consecutive output instances
// [gfirst[g], gfirst[g+1]) read the same A instance (group g).
struct StepDesc {
    const float2 *A;
    const float2 *B;
    float2 *C;
    int64_t sA, sB, sC;           // elements per instance
    const int32_t *sigA, *sigB;   // [n_sig]
    const int32_t *outA, *outB;   // [nOut]
    int32_t nOutA, nOutB, nOut;
    int32_t sched;                // schedule variant of the step's kernel (0 or 1; the autotuner's choice)
    int32_t tc_resident_b;        // tensor cores: keep B resident in shared memory where it fits
    int32_t tc_pair;              // tensor cores: BF16x3 packed B, schedule 0, N >= 64, K >= 256: column tiles in pairs (N = 256 MMAs)
    int32_t pad_;
    int64_t nInst;
    int64_t nInstB;               // B instances (tensor-core B dictionary)
    const int32_t *EA, *EB;       // accumulated exponents of the operands
    int32_t *EC;
    const uint32_t *mxA, *mxB;    // max-|component| bits of the operands (null: no rescale)
    uint32_t *mxC;                // max-|component| bits of C (null: not tracked)
    int32_t mb, kb, nb;
    int32_t max_group;            // largest group (instances)
    const int64_t *gfirst;        // [n_groups + 1]
    int64_t n_groups;
    const int64_t *ctab;          // non-empty column tiles: (group << 20) | tile of 64 columns
    int64_t n_ctab;
    const int4 *trec;             // per column tile: {first instance, count, A instance, first column}
    const int2 *ptab;             // N = 64: per column tile with groups padded to even counts,
                                  // {group's first column tile, its first padded one} (else null)
    int64_t n_ptab;
    const int2 *instab;           // per output instance: {A instance, B instance}
    uint8_t *bpack;               // tensor cores: scratch for B packed in MMA form (null: none)
    int64_t bpack_bytes;
    int8_t pAm[40];
    int8_t pBn[24];
    int8_t pCm[40];
    int8_t pCn[24];
};

struct FillJobD {
    int64_t dst, src;
    int32_t leaf_high, n;
};

struct LeafHighD {
    int32_t cnt;
    int32_t j[4];
    int32_t stride[4];
};

// Launchers return cudaGetLastError() of the launch.
cudaError_t launch_fill(const FillJobD *jobs, int64_t njobs, const LeafHighD *highs, int64_t batch,
                        float2 *ws, cudaStream_t s);
cudaError_t launch_step_row(const StepDesc &d, cudaStream_t s);
cudaError_t launch_step_gemm_simt(const StepDesc &d, cudaStream_t s);
// Steps with M N <= 4 outputs per instance and K >= 64: one block per
// output, a dot product of two K-contiguous runs (FP32).
cudaError_t launch_step_dot(const StepDesc &d, cudaStream_t s);
// One-time per-device setup of the SIMT GEMM (its dynamic shared memory).
cudaError_t init_simt_kernels();
// The root holds 2^r entries per instance (r open output qubits, its bit t
// the t-th lowest); row p's completion x (most significant bit: the lowest
// open qubit) is root entry bit-reverse_r(x).
cudaError_t launch_accumulate(const float2 *root, const int32_t *E, const int32_t *uniq, int64_t k,
                              int64_t n_sig, int32_t n_out, int r, double *amps, cudaStream_t s);
cudaError_t launch_extract(const float2 *root, const int32_t *E, const int32_t *uniq, int64_t k,
                           int64_t sigma, int32_t n_out, int r, double *out, cudaStream_t s);
cudaError_t launch_xeb(const double *amps, int64_t k, double scale, double *out, cudaStream_t s);
cudaError_t launch_pt_moments(const double *amps, int64_t k, double n_states, double fid, double *out,
                              cudaStream_t s);
cudaError_t launch_sample(const double *amps, int64_t k, int r, const double *uniform, int64_t *picks,
                          cudaStream_t s);
// FP32 FMA throughput probe: `blocks` blocks of 256 threads, each thread
// 16 * iters flops; out (>= blocks floats) is written only in a case that
// does not occur.
cudaError_t launch_fma_probe(int64_t blocks, int64_t iters, float *out, cudaStream_t s);
cudaError_t launch_pt_hist(const double *amps, int64_t k, double n_states, double x_max, int nbins,
                           unsigned long long *counts, cudaStream_t s);

// Tensor-core path (gemm_tc.cu).  precision: 1 = TF32, 2 = BF16x3.
// Returns cudaErrorNotSupported for shapes it does not take.
bool gemm_tc_supports(const StepDesc &d);
// A tensor-core step keeps B resident in shared memory (schedule 0: a
// group's whole B; schedule 1: one column tile's) when it fits: the chunk
// count, else 0.
int tc_resident_b_chunks(const StepDesc &d);
// Schedule 0 of a tensor-core step whose B instances all fit one 64-column
// tile keeps them resident for the whole launch (a dictionary): the chunk
// count, else 0.
int tc_dictionary_chunks(const StepDesc &d);
// Bytes of the packed-B form of a step (every B instance in the MMA layout,
// 16 KB per 64 columns x 16 complex k), 0 if the step cannot take it.
int64_t tc_packed_b_bytes(const StepDesc &d);
// One-time per-device setup (function attributes, SM count); call outside
// any stream capture.
cudaError_t init_kernels();
// TMA descriptor of a step's A operand (n_inst_a instances); encoded on the
// host once the workspace is bound.
cudaError_t make_a_map(const StepDesc &d, int64_t n_inst_a, CUtensorMap *map);
cudaError_t launch_step_gemm_tc(const StepDesc &d, const CUtensorMap *a_map, int precision, int32_t *err_flag,
                                cudaStream_t s);

// Fused chain of small-operand steps (chain.cu); the planner's Chain as the
// kernel sees it.
constexpr int CH_MAXL = 6;    // steps
constexpr int CH_MAXT = 10;   // tile bits
constexpr int CH_MAXO = 40;   // outside bits
constexpr int CH_MAX_SMEM = 160 * 1024;
struct ChainDesc {
    const float2 *A;              // A_1
    float2 *C;                    // C_L
    int64_t sA, sC;               // elements per instance
    const float2 *B[CH_MAXL];     // B_j, 2^(kb_j + nb_j) elements per instance
    const uint32_t *mxA, *mxB[CH_MAXL];  // max-|component| words (null: no rescale)
    uint32_t *mxC;
    const int32_t *EA, *EB[CH_MAXL];
    int32_t *EC;
    const int32_t *tab;           // per C_L instance: a_1, b_1 .. b_L
    const unsigned char *idx;     // index tables (plan.hpp, Chain::off_idx)
    int64_t n_inst;               // C_L instances
    int64_t oblocks;              // blocks per instance (set by the launcher)
    int32_t L, tin, no, tmax;     // steps, A_1 tile bits, outside bits, largest tile bits
    int32_t kb[CH_MAXL], nb[CH_MAXL], tb[CH_MAXL];
    int8_t code[CH_MAXL][CH_MAXT];      // per output tile bit: 0x80 | n bit, or A tile bit
    int8_t in_pos[CH_MAXT], out_pos[CH_MAXT];
    int8_t o_in[CH_MAXO], o_out[CH_MAXO];
};
size_t chain_smem_bytes(const ChainDesc &d);
cudaError_t init_chain_kernel();
cudaError_t launch_chain(ChainDesc d, cudaStream_t s);

// Cost-model MLP (mlp.cu); sizes and parameter layout in include/tn.h.
size_t mlp_grad_scratch_bytes(int64_t n);
cudaError_t mlp_forward(const float *params, const float *X, int64_t n, float *y, cudaStream_t s);
cudaError_t mlp_grad(const float *params, const float *X, const float *t, int64_t n, float *grad, float *loss,
                     float *scratch, cudaStream_t s);
cudaError_t mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr, float beta1,
                     float beta2, float eps, cudaStream_t s);
cudaError_t mlp_to_half(const float *params, uint16_t *params16, cudaStream_t s);
cudaError_t mlp_forward_f16(const uint16_t *params16, const float *X, int64_t n, float *y, cudaStream_t s);

}  // namespace tnk
