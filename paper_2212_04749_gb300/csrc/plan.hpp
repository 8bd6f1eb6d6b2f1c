// Host-side plan of a multiple-amplitude contraction (no CUDA calls here).
//
// The plan turns (circuit, bitstrings, contraction tree, sliced edges) into
//   * the fused tensor network (SM Sec. II: one tensor per two-qubit gate),
//   * the static reuse-instance DAG: for every tree node, the distinct
//     projections of the bitstrings onto the node's output qubits (the width
//     w of the paper's reuse tree, main text Eq. (1) and SM Sec. III),
//     times the values of the sliced edges inside the node that run side by
//     side in one pass,
//   * a step list (one pairwise contraction per internal node) in
//     execution order, split into slice-independent steps (run once per
//     call) and slice-dependent steps (run once per slice batch),
//   * a workspace layout (byte offsets into one caller-owned device buffer).
#pragma once

#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tn.h"

namespace tnp {

using cd = std::complex<double>;

enum LegKind { LEG_BOND = 0, LEG_OUT = 1, LEG_FIXED = 2 };

struct Leg {
    int kind;
    int id;  // bond edge id, or qubit for an output leg
};

// Fused tensor of one two-qubit gate; t[((oa*2+ob)*2+ia)*2+ib], the legs
// in that order.  A LEG_FIXED input leg is |0>: only ia = 0 (ib = 0) holds
// the absorbed input vector.
struct LeafTensor {
    int gate;
    int qa, qb;
    Leg legs[4];  // oa, ob, ia, ib
    cd t[16];
};

struct Network {
    int n_qubits = 0, n_tensors = 0, n_edges = 0;
    std::vector<LeafTensor> leaves;
    std::vector<std::array<int, 2>> edge_ends;
    std::vector<int> out_tensor;  // per qubit
};

bool build_network(const tn_circuit *circ, Network &net, std::string &err);

// Device-side workspace offsets (bytes) of one node's data.
struct NodeBuf {
    int64_t data = -1;  // complex64 [n_inst][2^rank]
    int64_t E = -1;     // int32 [n_inst] accumulated power-of-two exponent
    int64_t mx = -1;    // uint32 [n_inst] max |component| float bits (rescale)
    int64_t sig = -1;   // int32 [n_sig] -> (sigL, sigR) packed as 2 arrays
    int64_t out = -1;   // int32 [n_out] -> (outL, outR) packed as 2 arrays
};

struct Node {
    int left = -1, right = -1;   // children (-1 for leaves)
    int parent = -1;
    std::vector<int> layout;     // open bond edges, bit 0 first
    std::vector<int> outs;       // output qubits in the subtree (sorted)
    std::vector<int> slices;     // internal sliced-edge indices t in the subtree (sorted)
    std::vector<int> slices_low; // those batched in one pass (t < m_low)
    uint64_t hmask = 0;          // looped sliced edges in the subtree (bit t - m_low)
    int level = 64;              // lowest bit of hmask; 64 = computed once per call
    bool persistent = false;     // buffer kept across slice batches
    int n_out = 1;               // distinct projections of the bitstrings on outs
    int64_t n_sig = 1;           // 2^{|slices_low|}
    int64_t n_inst = 1;          // n_sig * n_out
    int rank = 0;
    // instance maps (internal nodes): out-instance -> child out-instances,
    // slice-instance -> child slice-instances
    std::vector<int32_t> outL, outR, sigL, sigR;
    // leaves: the projection value (2 bits: oa, ob order) of each out-instance
    std::vector<int32_t> leaf_outval;
    NodeBuf buf;
    int step = -1;               // step producing this node
    int last_use = -1;           // last step reading it
};

// One pairwise contraction C = A (x) B over K = I_A n I_B.
// A is the operand with more entries per instance.  Output layout: the free
// bits of B (in B's order) at the bottom, then the free bits of A.
struct Step {
    int node = -1, a = -1, b = -1;
    int mb = 0, kb = 0, nb = 0;
    std::vector<int8_t> pAm, pAk, pBk, pBn;  // bit positions in A / B
    std::vector<int8_t> pCm, pCn;            // positions of the m / n bits in C
    int level = 64;          // recomputed in batch b > first iff level <= ctz(b)
    double runs = 1;         // passes over all 2^h batches
    int64_t n_groups = 0;    // runs of consecutive output instances sharing an A instance
    std::vector<int64_t> group_first;  // n_groups + 1 boundaries
    int64_t off_groups = -1;           // workspace offset of group_first
    std::vector<int64_t> col_tiles;    // non-empty (group, 64-column tile) pairs: g * 2^20 + tile
    int64_t off_col_tiles = -1;
    int64_t off_tile_rec = -1;         // per column tile: {first instance, count, A instance, first column}
    int64_t off_inst_ab = -1;          // per output instance: {A instance, B instance} (int32 pairs)
    // N = 64 (one column tile per instance): column tiles with every group
    // padded to an even count, for the tensor cores' column-tile pairs;
    // per padded tile {the group's first column tile, its first padded one}
    int64_t n_pair_tiles = 0;
    int64_t off_pair_tab = -1;
    int kernel = 0;          // 0 = per-row SIMT, 1 = tiled SIMT GEMM, 2 = tensor-core GEMM
    int chain = -1;          // fused chain holding this step (-1: none)
    bool chain_last = false; // the chain runs at its last step; the others launch nothing
    double flops = 0;        // executed per pass: 8 * n_inst * 2^{mb+kb+nb}
    double bytes = 0;        // A + B reads and C write per pass
};

// A fused chain (SM Sec. V.C): steps s_1..s_L where each step's A operand is
// the previous step's output, instance counts do not grow, and every side
// operand B_j is small.  It runs as one kernel at s_L: per output instance
// and per value of the "outside" bits O (A_1's free bits that no chain step
// touches), a tile of A_1 (its other bits) is loaded once, multiplied by
// B_1 .. B_L in shared memory, and written to C_L; the intermediates
// C_1 .. C_{L-1} are never stored.
constexpr int CHAIN_MAX_STEPS = 6;
constexpr int CHAIN_MAX_TILE_BITS = 10;
struct Chain {
    std::vector<int> steps;            // s_1 .. s_L
    int tin = 0;                       // tile bits of A_1
    int no = 0;                        // outside bits
    std::vector<int> tbits;            // tile bits of C_j, j = 1..L
    std::vector<int8_t> in_pos;        // address bit in A_1 of each A_1 tile bit (ascending)
    std::vector<int8_t> o_in_pos, o_out_pos;  // address bit of each outside bit in A_1 and C_L
    std::vector<int8_t> out_pos;       // address bit in C_L of each C_L tile bit (ascending)
    std::vector<std::vector<int8_t>> code;  // per step, per output tile bit: 0x80|i (n bit i) or r (A tile bit r)
    int64_t off_tab = -1;              // int32 per C_L instance: a_1, b_1 .. b_L
    // index tables, uploaded at off_idx (int64 inoff[2^tin], int64
    // outoff[2^tL], then per step int32 rowin[R_j], rowout[R_j], colout[N_j]):
    // address offset in A_1 of each input tile entry, in C_L of each output
    // tile entry, and per step the input / output tile index of each row
    // (R_j = 2^(tbits_j - nb_j)) and the output tile bits of each column
    std::vector<int64_t> inoff, outoff;
    std::vector<std::vector<int32_t>> rowin, rowout, colout;
    int64_t off_idx = -1;
};

struct Plan {
    Network net;
    tn_options opt{};
    int n_qubits = 0;
    int64_t k = 0;                    // input rows
    std::vector<int32_t> uniq_of;     // input row -> distinct bitstring id
    int64_t k_unique = 0;
    std::vector<std::vector<uint8_t>> ubits;  // distinct bitstrings (0 at open qubits)
    std::vector<int> open_qubits;     // output qubits left open, ascending; the root's bit t is open_qubits[t]
    std::vector<int> sliced;          // sliced edge ids, external order (j-th takes bit j of s)
    std::vector<int> perm;            // internal slice index t -> external j
    int m_low = 0;                    // sliced edges batched in one pass
    int64_t n_batches = 1;
    std::vector<Node> nodes;          // 2T-1
    std::vector<Step> steps;          // SSA order
    std::vector<Chain> chains;        // fused chains (opt.fuse)
    int n_static_steps = 0;
    int root = -1;
    int max_rank = 0;
    double flops_ma = 0, flops_sa = 0, flops_exec = 0, bytes_min = 0;
    int64_t peak_tensor_bytes = 0;

    // workspace layout
    int64_t ws_bytes = 0;
    int64_t off_leaf_full = -1;       // complex64 full leaf tensors
    int64_t off_fill_jobs = -1;       // FillJob table
    int64_t n_fill_jobs = 0;
    int64_t off_leaf_high = -1;       // LeafHigh table
    int64_t off_uniq = -1;            // int32 [k] input row -> root out-instance
    int64_t off_emax = -1, emax_bytes = 0;  // max words of every node, by level
    std::vector<int64_t> emax_prefix;       // [lv]: bytes covering the nodes of level <= lv
    int64_t off_scratch = -1;               // 256 bytes of device scratch (error word)
    int64_t off_bpack = -1, bpack_bytes = 0; // tensor cores: room for one step's B packed in MMA form
    // host images uploaded at bind time: (offset, bytes)
    std::vector<std::pair<int64_t, std::vector<uint8_t>>> uploads;
};

struct FillJob {          // one leaf instance block
    int64_t dst;          // complex64 element offset of the block in the workspace
    int64_t src;          // element offset in the full-leaf region, high-slice bits = 0
    int32_t leaf_high;    // index into the LeafHigh table
    int32_t n;            // elements
};

struct LeafHigh {         // sliced legs of a leaf that vary across batches
    int32_t cnt;
    int32_t j[4];         // high sliced index (j - m_low)
    int32_t stride[4];    // element stride of that leg in the full-leaf block
};

bool make_plan(const tn_circuit *circ, const uint8_t *bits, int64_t k, const int32_t *ssa,
               const int32_t *sliced, int32_t n_sliced, const tn_options *opt, Plan &plan,
               std::string &err, int &code);

}  // namespace tnp
