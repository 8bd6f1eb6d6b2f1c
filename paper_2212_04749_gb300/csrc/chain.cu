// Fused chain of small-operand steps (SM Sec. V.C: a tile of the big tensor
// stays in fast memory while the chain's small tensors are applied to it,
// and only the chain's last output is written back).
//
// Chain s_1 .. s_L:  C_j(m, n) = sum_k C_{j-1}(k, m) B_j(k, n), C_0 = A_1.
// Bits of A_1 that no chain step contracts (the outside bits O) pass
// through to C_L unchanged; for each output instance and each value o of
// O the kernel
//   1. loads the A_1 tile (A_1's other bits: 2^tin entries) into the
//      warp's shared-memory buffer,
//   2. applies B_1 .. B_L (staged once per block in shared memory) tile to
//      tile, ping-ponging between two buffers of 2^dt entries,
//   3. scales by the operands' power-of-two factors and writes the C_L tile
//      through its address bits.
// Tile index bits are the tile's address bits in ascending order, so the
// contracted bits of every step are the lowest bits of its input tile (the
// planner keeps every operand K-major) and an output element (m, n) reads
// input entries base(m) + k, k < K.  Address offsets and index maps come from
// per-block tables; a lane keeps one input row in registers and walks the
// columns with B broadcast from shared memory.
//
// Rescale: the intermediates are not rescaled (the chain is short and the
// operands come normalised); C_L is multiplied by 2^-(ea + sum_j eb_j), the
// exponents of the operands' largest components, and its exponent is
// E_A + ea + sum_j (E_Bj + eb_j).  Power-of-two factors are exact.
#include "kernels.cuh"

namespace tnk {

namespace {

constexpr int CH_THREADS = 256;
constexpr int CH_WARPS = CH_THREADS / 32;
constexpr int CH_OPW = 64;  // outside values per warp and block

__device__ __forceinline__ int ch_exp(uint32_t bits) {
    if (bits == 0u) return 0;
    const int e = int((bits >> 23) & 0xffu) - 127;
    return max(-126, min(126, e));
}

__device__ __forceinline__ float ch_pow2(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ void ch_record_max(uint32_t *slot, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(slot), "r"(v) : "memory");
}

// Shared memory (dynamic): B_1 .. B_L | per-warp tile buffers.  Index
// tables, built by the planner and read through the L1 cache:
//   inoff[e]    address offset in A_1 of input tile entry e
//   outoff[t]   address offset in C_L of output tile entry t
//   per step j: rowin[r]  input tile index of row r's first k (k = 0)
//               rowout[r] output tile index of row r at n = 0
//               colout[n] output tile bits of column n
// Rows r enumerate the step's output tile bits that come from A (its m bits
// inside the tile), columns n its n bits, so out(r, n) = sum_k in(rowin[r]
// + k) B_j(k, n) and is stored at rowout[r] | colout[n].
struct ChTables {
    const int64_t *inoff, *outoff;
    const int32_t *rowin[CH_MAXL], *rowout[CH_MAXL], *colout[CH_MAXL];
};

// Tile buffers are XOR-swizzled: entry i lives at i ^ ((i >> 4) & 15), so
// lanes that walk different rows (row stride 8 or 16 entries) hit
// different banks.
__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }

__device__ __forceinline__ void cmac(float &re, float &im, float2 u, float2 v) {
    re = fmaf(u.x, v.x, re);
    re = fmaf(-u.y, v.y, re);
    im = fmaf(u.x, v.y, im);
    im = fmaf(u.y, v.x, im);
}

__global__ void __launch_bounds__(CH_THREADS) k_chain(const ChainDesc d) {
    extern __shared__ __align__(16) unsigned char ch_raw[];
    __shared__ int64_t s_boff[CH_MAXL];
    __shared__ int32_t s_rows[CH_MAXL];
    __shared__ float s_sc;
    __shared__ uint32_t s_mx;
    __shared__ int32_t s_tab[CH_MAXL + 1], s_e[CH_MAXL + 1], s_E[CH_MAXL + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t inst = int64_t(blockIdx.x) / d.oblocks;
    const int64_t ob = int64_t(blockIdx.x) % d.oblocks;
    const int L = d.L;
    if (tid <= L) s_tab[tid] = d.tab[inst * (L + 1) + tid];
    if (tid == 0) {
        int64_t o = 0;
        for (int j = 0; j < L; ++j) {
            s_boff[j] = o;
            o += int64_t(1) << (d.kb[j] + d.nb[j]);
            s_rows[j] = 1 << (d.tb[j] - d.nb[j]);
        }
        s_mx = 0u;
    }
    __syncthreads();
    // index tables (global, read through the L1 cache)
    ChTables tb;
    {
        const unsigned char *q = d.idx;
        tb.inoff = reinterpret_cast<const int64_t *>(q);
        q += size_t(8) << d.tin;
        tb.outoff = reinterpret_cast<const int64_t *>(q);
        q += size_t(8) << d.tb[L - 1];
        for (int j = 0; j < L; ++j) {
            tb.rowin[j] = reinterpret_cast<const int32_t *>(q);
            q += size_t(4) << (d.tb[j] - d.nb[j]);
            tb.rowout[j] = reinterpret_cast<const int32_t *>(q);
            q += size_t(4) << (d.tb[j] - d.nb[j]);
            tb.colout[j] = reinterpret_cast<const int32_t *>(q);
            q += size_t(4) << d.nb[j];
        }
    }
    const int64_t bsz = s_boff[L - 1] + (int64_t(1) << (d.kb[L - 1] + d.nb[L - 1]));
    float2 *Bs = reinterpret_cast<float2 *>(ch_raw);
    float2 *X0 = Bs + ((bsz + 1) & ~int64_t(1)) + int64_t(warp) * 2 * (int64_t(1) << d.tmax);
    float2 *X1 = X0 + (int64_t(1) << d.tmax);
    // operand exponents: thread q <= L loads those of operand q (A_1, B_q)
    if (tid <= L) {
        const int id = s_tab[tid];
        const uint32_t *mx = tid == 0 ? d.mxA : d.mxB[tid - 1];
        const int32_t *E = tid == 0 ? d.EA : d.EB[tid - 1];
        const int e = mx ? ch_exp(__ldg(mx + id)) : 0;
        s_e[tid] = e;
        s_E[tid] = __ldg(E + id) + e;
    }
    __syncthreads();
    if (tid == 0) {
        float sc = 1.f;
        int ec = 0;
        for (int q = 0; q <= L; ++q) {
            sc *= ch_pow2(-s_e[q]);
            ec += s_E[q];
        }
        s_sc = sc;
        if (ob == 0) d.EC[inst] = ec;
    }
    // stage B_1 .. B_L of this instance
    for (int j = 0; j < L; ++j) {
        const int kn = 1 << (d.kb[j] + d.nb[j]);
        const float2 *src = d.B[j] + int64_t(s_tab[1 + j]) * kn;
        float2 *dst = Bs + s_boff[j];
        for (int e = tid; e < kn; e += CH_THREADS) dst[e] = __ldg(src + e);
    }
    __syncthreads();
    const float sc = s_sc;
    const int64_t n_o = int64_t(1) << d.no;
    const int a = s_tab[0];
    uint32_t lmax = 0u;
    for (int qo = 0; qo < CH_OPW; ++qo) {
        const int64_t o = ob * (CH_WARPS * CH_OPW) + int64_t(qo) * CH_WARPS + warp;
        if (o >= n_o) break;  // uniform per warp
        int64_t abase = int64_t(a) * d.sA, cbase = inst * d.sC;
        for (int b = 0; b < d.no; ++b)
            if ((o >> b) & 1) {
                abase += int64_t(1) << d.o_in[b];
                cbase += int64_t(1) << d.o_out[b];
            }
        // 1. the A_1 tile by cp.async (every load in flight at once, no
        // register round trip)
        for (int e = lane; e < (1 << d.tin); e += 32) {
            const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(X0 + swz(e)));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(d.A + abase + __ldg(tb.inoff + e))
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        // 2. B_1 .. B_L: work items (row, block of cpi columns) over the
        // lanes; a lane keeps its row's K inputs in registers and walks its
        // columns with B read as a warp broadcast
        float2 *xi = X0, *xo = X1;
        for (int j = 0; j < L; ++j) {
            const int K = 1 << d.kb[j], N = 1 << d.nb[j], rows = s_rows[j];
            int cpi = (rows * N) / 32;  // columns per item, a power of two in [1, N]
            cpi = cpi < 1 ? 1 : (cpi > N ? N : cpi);
            const int cb = N / cpi, items = rows * cb;
            const float2 *Bj = Bs + s_boff[j];
            const int32_t *rin = tb.rowin[j], *rout = tb.rowout[j], *cout = tb.colout[j];
            for (int it = lane; it < items; it += 32) {
                const int r = it / cb, n0 = (it - r * cb) * cpi;
                const int ib = __ldg(rin + r), obase = __ldg(rout + r);
                if (K <= 16) {
                    float2 x[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) x[k] = k < K ? xi[swz(ib + k)] : make_float2(0.f, 0.f);
                    for (int n = n0; n < n0 + cpi; ++n) {
                        const float2 *bc = Bj + n * K;
                        float re = 0.f, im = 0.f;
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (k < K) cmac(re, im, x[k], bc[k]);
                        xo[swz(obase | __ldg(cout + n))] = make_float2(re, im);
                    }
                } else {
                    for (int n = n0; n < n0 + cpi; ++n) {
                        const float2 *bc = Bj + n * K;
                        float re = 0.f, im = 0.f;
                        for (int k = 0; k < K; ++k) cmac(re, im, xi[swz(ib + k)], bc[k]);
                        xo[swz(obase | __ldg(cout + n))] = make_float2(re, im);
                    }
                }
            }
            __syncwarp();
            float2 *tmp = xi;
            xi = xo;
            xo = tmp;
        }
        // 3. scale and write the C_L tile
        for (int t = lane; t < (1 << d.tb[L - 1]); t += 32) {
            const float2 u = xi[swz(t)];
            const float2 v = make_float2(u.x * sc, u.y * sc);
            d.C[cbase + __ldg(tb.outoff + t)] = v;
            lmax = max(lmax, __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))));
        }
        __syncwarp();  // the buffers are rewritten for the next outside value
    }
    if (d.mxC) {
        const uint32_t wmax = __reduce_max_sync(0xffffffffu, lmax);
        if (lane == 0 && wmax) atomicMax(&s_mx, wmax);
        __syncthreads();
        if (tid == 0 && s_mx) ch_record_max(d.mxC + inst, s_mx);
    }
}

}  // namespace

size_t chain_smem_bytes(const ChainDesc &d) {
    size_t b = 0;
    for (int j = 0; j < d.L; ++j) b += size_t(1) << (d.kb[j] + d.nb[j]);
    b = (b + 1) & ~size_t(1);  // the tile buffers start 16-byte aligned
    b += size_t(CH_WARPS) * 2 * (size_t(1) << d.tmax);
    return b * sizeof(float2);
}

cudaError_t init_chain_kernel() {
    return cudaFuncSetAttribute(k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, CH_MAX_SMEM);
}

cudaError_t launch_chain(ChainDesc d, cudaStream_t s) {
    if (d.L < 1 || d.L > CH_MAXL || d.tmax > CH_MAXT || d.no > CH_MAXO) return cudaErrorInvalidValue;
    const size_t smem = chain_smem_bytes(d);
    if (smem > size_t(CH_MAX_SMEM)) return cudaErrorInvalidValue;
    const int64_t n_o = int64_t(1) << d.no;
    d.oblocks = (n_o + CH_WARPS * CH_OPW - 1) / (CH_WARPS * CH_OPW);
    const int64_t blocks = d.n_inst * d.oblocks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_chain<<<dim3((unsigned)blocks), CH_THREADS, smem, s>>>(d);
    return cudaGetLastError();
}

}  // namespace tnk
