// C ABI of the contraction library (declared in include/tn.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <tuple>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tn.h"
#include "kernels.cuh"
#include "plan.hpp"

namespace {

thread_local std::string g_err;

int set_err(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_err(TN_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

struct PlanObj {
    tnp::Plan P;
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<tnk::StepDesc> desc;  // per step
    struct alignas(64) AMap {
        CUtensorMap map;
        bool ok;
    };
    std::vector<AMap> amap;           // per step: TMA descriptor of A (tensor-core steps)
    std::vector<tnk::ChainDesc> chain_desc;  // per fused chain
    int32_t *err_flag = nullptr;      // device word for bounded waits
    bool tc_resident_b = true;        // tensor-core GEMM keeps B in shared memory where it fits
    bool tc_pair = true;              // tensor-core GEMM: column-tile pairs (N = 256 MMAs) where packed B allows
    bool profile = false;
    std::vector<cudaEvent_t> ev;          // pool, two per profiled launch
    std::vector<int> ev_step;             // step of each recorded pair
    size_t ev_used = 0;
    std::vector<int32_t> step_kernel;     // kernel family each step ran last (0 row, 1 SIMT GEMM, 2 TC GEMM)
    std::vector<int32_t> config_override; // per step: -1 plan choice, else a configuration (tn.h)
    std::vector<uint8_t> chain_on;        // per fused chain: run as one kernel (1) or as its steps (0)
    bool chain_fused(int c) const { return c >= 0 && (c >= (int)chain_on.size() || chain_on[c] != 0); }
    struct GraphKey {
        int precision;
        int64_t lo, hi;
        const double *amps;
        bool operator<(const GraphKey &o) const {
            return std::tie(precision, lo, hi, amps) < std::tie(o.precision, o.lo, o.hi, o.amps);
        }
    };
    std::map<GraphKey, cudaGraphExec_t> graphs;  // captured tn_contract launch sequences
    cudaStream_t cap_stream = nullptr;           // private stream the sequences are captured on
    void drop_graphs() {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
    }
    int64_t last_batches = 0;
};

template <class T>
T *at(PlanObj *o, int64_t off) {
    return reinterpret_cast<T *>(o->ws + off);
}

void build_descs(PlanObj *o) {
    tnp::Plan &P = o->P;
    o->desc.clear();
    for (const tnp::Step &st : P.steps) {
        const tnp::Node &nd = P.nodes[st.node];
        const tnp::Node &A = P.nodes[st.a], &B = P.nodes[st.b];
        tnk::StepDesc d;
        std::memset(&d, 0, sizeof(d));
        d.A = at<const float2>(o, A.buf.data);
        d.B = at<const float2>(o, B.buf.data);
        d.C = at<float2>(o, nd.buf.data);
        d.sA = int64_t(1) << A.rank;
        d.sB = int64_t(1) << B.rank;
        d.sC = int64_t(1) << nd.rank;
        const bool a_left = (st.a == nd.left);
        const int32_t *sig = at<const int32_t>(o, nd.buf.sig);
        const int32_t *out = at<const int32_t>(o, nd.buf.out);
        d.sigA = a_left ? sig : sig + nd.n_sig;
        d.sigB = a_left ? sig + nd.n_sig : sig;
        d.outA = a_left ? out : out + nd.n_out;
        d.outB = a_left ? out + nd.n_out : out;
        d.nOutA = A.n_out;
        d.nOutB = B.n_out;
        d.nOut = nd.n_out;
        d.nInst = nd.n_inst;
        d.nInstB = B.n_inst;
        d.EA = at<const int32_t>(o, A.buf.E);
        d.EB = at<const int32_t>(o, B.buf.E);
        d.EC = at<int32_t>(o, nd.buf.E);
        const bool rs = P.opt.rescale != 0;
        d.mxA = rs ? at<const uint32_t>(o, A.buf.mx) : nullptr;
        d.mxB = rs ? at<const uint32_t>(o, B.buf.mx) : nullptr;
        d.mxC = rs ? at<uint32_t>(o, nd.buf.mx) : nullptr;
        d.mb = st.mb;
        d.kb = st.kb;
        d.nb = st.nb;
        for (int j = 0; j < st.mb; ++j) {
            d.pAm[j] = st.pAm[j];
            d.pCm[j] = st.pCm[j];
        }
        for (int j = 0; j < st.nb; ++j) {
            d.pBn[j] = st.pBn[j];
            d.pCn[j] = st.pCn[j];
        }
        d.gfirst = at<const int64_t>(o, st.off_groups);
        d.n_groups = st.n_groups;
        d.ctab = at<const int64_t>(o, st.off_col_tiles);
        d.n_ctab = (int64_t)st.col_tiles.size();
        d.trec = at<const int4>(o, st.off_tile_rec);
        d.ptab = st.n_pair_tiles > 0 ? at<const int2>(o, st.off_pair_tab) : nullptr;
        d.n_ptab = st.n_pair_tiles;
        d.instab = at<const int2>(o, st.off_inst_ab);
        d.bpack = P.bpack_bytes > 0 ? at<uint8_t>(o, P.off_bpack) : nullptr;
        d.bpack_bytes = P.bpack_bytes;

        int64_t mg = 0;
        for (int64_t g = 0; g < st.n_groups; ++g) mg = std::max(mg, st.group_first[g + 1] - st.group_first[g]);
        d.max_group = (int32_t)mg;
        o->desc.push_back(d);
    }
    // fused chains
    o->chain_desc.clear();
    for (const tnp::Chain &c : P.chains) {
        tnk::ChainDesc cd;
        std::memset(&cd, 0, sizeof(cd));
        const int L = (int)c.steps.size();
        const tnp::Step &s1 = P.steps[c.steps[0]], &sL = P.steps[c.steps[L - 1]];
        const tnp::Node &A1 = P.nodes[s1.a], &CL = P.nodes[sL.node];
        const bool rs = P.opt.rescale != 0;
        cd.A = at<const float2>(o, A1.buf.data);
        cd.C = at<float2>(o, CL.buf.data);
        cd.sA = int64_t(1) << A1.rank;
        cd.sC = int64_t(1) << CL.rank;
        cd.mxA = rs ? at<const uint32_t>(o, A1.buf.mx) : nullptr;
        cd.mxC = rs ? at<uint32_t>(o, CL.buf.mx) : nullptr;
        cd.EA = at<const int32_t>(o, A1.buf.E);
        cd.EC = at<int32_t>(o, CL.buf.E);
        cd.tab = at<const int32_t>(o, c.off_tab);
        cd.idx = at<const unsigned char>(o, c.off_idx);
        cd.n_inst = CL.n_inst;
        cd.L = L;
        cd.tin = c.tin;
        cd.no = c.no;
        cd.tmax = c.tin;
        for (int j = 0; j < L; ++j) {
            const tnp::Step &st = P.steps[c.steps[j]];
            const tnp::Node &B = P.nodes[st.b];
            cd.B[j] = at<const float2>(o, B.buf.data);
            cd.mxB[j] = rs ? at<const uint32_t>(o, B.buf.mx) : nullptr;
            cd.EB[j] = at<const int32_t>(o, B.buf.E);
            cd.kb[j] = st.kb;
            cd.nb[j] = st.nb;
            cd.tb[j] = c.tbits[j];
            cd.tmax = std::max(cd.tmax, c.tbits[j]);
            for (int b = 0; b < c.tbits[j]; ++b) cd.code[j][b] = c.code[j][b];
        }
        for (int b = 0; b < c.tin; ++b) cd.in_pos[b] = c.in_pos[b];
        for (size_t b = 0; b < c.out_pos.size(); ++b) cd.out_pos[b] = c.out_pos[b];
        for (int b = 0; b < c.no; ++b) {
            cd.o_in[b] = c.o_in_pos[b];
            cd.o_out[b] = c.o_out_pos[b];
        }
        o->chain_desc.push_back(cd);
    }
    // TMA descriptors of the A operands, for every step the tensor-core
    // kernel can take (it may be chosen at run time)
    o->amap.assign(P.steps.size(), PlanObj::AMap{});
    for (size_t s = 0; s < P.steps.size(); ++s) {
        const tnk::StepDesc &d = o->desc[s];
        o->amap[s].ok = tnk::gemm_tc_supports(d) &&
                        tnk::make_a_map(d, P.nodes[P.steps[s].a].n_inst, &o->amap[s].map) == cudaSuccess;
    }
}

// Configurations (tn.h): 0, 1 per-row kernel (schedule 0, 1); 2, 3 grouped
// GEMM (schedule 0, 1).
bool config_allowed(const tnp::Step &S, int c) {
    if (c < 0 || c >= TN_NCONFIG) return false;
    return c >= 2 || (S.nb <= 4 && S.kb + S.nb <= 8);
}

int effective_config(const PlanObj *o, int s) {
    if (s < (int)o->config_override.size() && o->config_override[s] >= 0) return o->config_override[s];
    return o->P.steps[s].kernel == 0 ? 0 : 2;
}

int run_step(PlanObj *o, int s, int precision, cudaStream_t st) {
    const tnp::Step &S = o->P.steps[s];
    if (o->chain_fused(S.chain)) {  // fused chain: runs whole at its last step
        if ((int)o->step_kernel.size() <= s) o->step_kernel.resize(o->P.steps.size(), -1);
        o->step_kernel[s] = 3;
        if (!S.chain_last) return TN_OK;
        const cudaError_t e = tnk::launch_chain(o->chain_desc[S.chain], st);
        if (e != cudaSuccess)
            return set_err(TN_ECUDA, "fused chain at step " + std::to_string(s) + ": " + cudaGetErrorString(e));
        return TN_OK;
    }
    const int cfg = effective_config(o, s);
    tnk::StepDesc d = o->desc[s];
    d.sched = cfg & 1;
    d.tc_resident_b = o->tc_resident_b ? 1 : 0;
    d.tc_pair = o->tc_pair ? 1 : 0;
    cudaError_t e;
    int fam;
    if (cfg < 2) {
        fam = 0;
        e = tnk::launch_step_row(d, st);
    } else if (d.mb + d.nb <= 2 && d.kb >= 6) {
        // a few long dot products per instance (e.g. the root): one block each
        fam = 1;
        e = tnk::launch_step_dot(d, st);
    } else if (precision != TN_FP32 && tnk::gemm_tc_supports(d)) {
        fam = 2;
        e = o->amap[s].ok ? tnk::launch_step_gemm_tc(d, &o->amap[s].map, precision, o->err_flag, st)
                          : cudaErrorInvalidValue;  // its TMA descriptor could not be encoded
    } else {
        fam = 1;
        e = tnk::launch_step_gemm_simt(d, st);
    }
    if ((int)o->step_kernel.size() <= s) o->step_kernel.resize(o->P.steps.size(), -1);
    o->step_kernel[s] = fam;
    if (e != cudaSuccess)
        return set_err(TN_ECUDA, "step " + std::to_string(s) + ": " + cudaGetErrorString(e));
    return TN_OK;
}

// Cost-model features of step s under configuration c (tn.h, TN_NFEAT).
void step_features(const tnp::Plan &P, int s, int precision, int c, float *f) {
    const tnp::Step &S = P.steps[s];
    const tnp::Node &nd = P.nodes[S.node], &A = P.nodes[S.a], &B = P.nodes[S.b];
    auto lg = [](double x) { return float(std::log2(x > 1.0 ? x : 1.0)); };
    auto run = [](const std::vector<int8_t> &pos) {
        int j = 0;
        while (j < (int)pos.size() && pos[j] == j) ++j;
        return j;
    };
    int crun = 0;  // lowest C address bits held by consecutive m bits
    while (crun < S.mb && S.pCm[crun] == crun) ++crun;
    tnk::StepDesc t;
    std::memset(&t, 0, sizeof(t));
    t.mb = S.mb;
    t.kb = S.kb;
    t.nb = S.nb;
    const bool gemm = c >= 2;
    const bool tc = gemm && precision != TN_FP32 && tnk::gemm_tc_supports(t);
    const double ng = double(S.n_groups > 0 ? S.n_groups : 1);
    int i = 0;
    f[i++] = S.mb / 32.f;
    f[i++] = S.kb / 32.f;
    f[i++] = S.nb / 32.f;
    f[i++] = A.rank / 32.f;
    f[i++] = B.rank / 32.f;
    f[i++] = lg(double(nd.n_inst)) / 32.f;
    f[i++] = lg(double(A.n_inst)) / 32.f;
    f[i++] = lg(double(B.n_inst)) / 32.f;
    f[i++] = lg(ng) / 32.f;
    f[i++] = lg(double(nd.n_inst) / ng * std::ldexp(1.0, S.nb)) / 32.f;
    f[i++] = run(S.pAm) / 32.f;
    f[i++] = run(S.pAk) / 32.f;
    f[i++] = run(S.pBk) / 32.f;
    f[i++] = run(S.pBn) / 32.f;
    f[i++] = crun / 32.f;
    f[i++] = lg(S.flops) / 64.f;
    f[i++] = lg(S.bytes) / 64.f;
    f[i++] = precision == TN_TF32 ? 1.f : 0.f;
    f[i++] = precision == TN_BF16X3 ? 1.f : 0.f;
    f[i++] = gemm ? 0.f : 1.f;
    f[i++] = tc ? 1.f : 0.f;
    f[i++] = gemm && !tc ? 1.f : 0.f;
    f[i++] = float(c & 1);
    f[i++] = lg(double(nd.n_inst) * std::ldexp(1.0, S.mb)) / 64.f;
}

// Batches [b_lo, b_hi) in order.  The first batch of the call runs every
// step; batch b > b_lo re-runs only the steps whose sliced edges changed
// from batch b-1 (level <= ctz(b)).  `per_batch(b)` runs after each batch.
template <class F>
int run_batches(PlanObj *o, int precision, int64_t b_lo, int64_t b_hi, cudaStream_t st, F per_batch) {
    tnp::Plan &P = o->P;
    const int nst = (int)P.steps.size();
    o->ev_used = 0;
    o->ev_step.clear();
    const auto *jobs = at<const tnk::FillJobD>(o, P.off_fill_jobs);
    const auto *highs = at<const tnk::LeafHighD>(o, P.off_leaf_high);
    for (int64_t b = b_lo; b < b_hi; ++b) {
        const int lv = (b == b_lo) ? 64 : __builtin_ctzll((unsigned long long)b);
        const int64_t clear = (b == b_lo) ? P.emax_bytes : P.emax_prefix[lv];
        if (clear) CU(cudaMemsetAsync(o->ws + P.off_emax, 0, clear, st));
        cudaError_t e = tnk::launch_fill(jobs, P.n_fill_jobs, highs, b, at<float2>(o, 0), st);
        if (e != cudaSuccess) return set_err(TN_ECUDA, std::string("leaf fill: ") + cudaGetErrorString(e));
        for (int s = 0; s < nst; ++s) {
            if (b != b_lo && P.steps[s].level > lv) continue;
            if (o->profile) {
                while (o->ev.size() < 2 * (o->ev_used + 1)) {
                    cudaEvent_t ev;
                    CU(cudaEventCreate(&ev));
                    o->ev.push_back(ev);
                }
                CU(cudaEventRecord(o->ev[2 * o->ev_used], st));
            }
            if (int rc = run_step(o, s, precision, st)) return rc;
            if (o->profile) {
                CU(cudaEventRecord(o->ev[2 * o->ev_used + 1], st));
                o->ev_step.push_back(s);
                o->ev_used++;
            }
        }
        if (int rc = per_batch(b)) return rc;
    }
    o->last_batches = b_hi - b_lo;
    (void)nst;
    return TN_OK;
}

// Fixed device scratch for tn_contract_static.  In host code this name is a
// host-side stand-in, not a device address: the address comes from
// cudaGetSymbolAddress, looked up once per device.
__device__ __align__(256) unsigned char g_static_scratch[TN_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
std::vector<void *> g_static_addr;  // per device ordinal; null until looked up

int static_scratch_address(void **out) {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_static_mu);
    if ((int)g_static_addr.size() <= dev) g_static_addr.resize(dev + 1, nullptr);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        CU(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return TN_OK;
}

}  // namespace

extern "C" {

const char *tn_last_error(void) { return g_err.c_str(); }

int tn_network(const tn_circuit *circ, int32_t *n_tensors, int32_t *n_edges, int32_t *edge_ends,
               int32_t *out_tensor) {
    tnp::Network net;
    std::string err;
    if (!tnp::build_network(circ, net, err)) return set_err(TN_EINVAL, err);
    if (n_tensors) *n_tensors = net.n_tensors;
    if (n_edges) *n_edges = net.n_edges;
    if (edge_ends)
        for (int e = 0; e < net.n_edges; ++e) {
            edge_ends[2 * e] = net.edge_ends[e][0];
            edge_ends[2 * e + 1] = net.edge_ends[e][1];
        }
    if (out_tensor)
        for (int q = 0; q < net.n_qubits; ++q) out_tensor[q] = net.out_tensor[q];
    g_err.clear();
    return TN_OK;
}

int tn_plan(const tn_circuit *circ, const uint8_t *bits, int64_t k, const int32_t *tree_ssa,
            const int32_t *sliced_edges, int32_t n_sliced, const tn_options *opt, tn_plan_t *out) {
    if (!out) return set_err(TN_EINVAL, "tn_plan: null output handle");
    *out = nullptr;
    std::unique_ptr<PlanObj> o(new PlanObj());
    std::string err;
    int code = TN_OK;
    try {
        if (!tnp::make_plan(circ, bits, k, tree_ssa, sliced_edges, n_sliced, opt, o->P, err, code))
            return set_err(code, err);
    } catch (const std::bad_alloc &) {
        return set_err(TN_ENOMEM, "tn_plan: host allocation failed");
    }
    *out = reinterpret_cast<tn_plan_t>(o.release());
    g_err.clear();
    return TN_OK;
}

int tn_plan_query(tn_plan_t plan, tn_plan_info *info) {
    if (!plan || !info) return set_err(TN_EINVAL, "tn_plan_query: null argument");
    const tnp::Plan &P = reinterpret_cast<PlanObj *>(plan)->P;
    std::memset(info, 0, sizeof(*info));
    info->n_tensors = P.net.n_tensors;
    info->n_edges = P.net.n_edges;
    info->n_nodes = (int32_t)P.nodes.size();
    info->n_steps = (int32_t)P.steps.size();
    info->n_unique = (int32_t)P.k_unique;
    info->n_sliced = (int32_t)P.sliced.size();
    info->slice_batch_log2 = P.m_low;
    info->n_batches = (int32_t)P.n_batches;
    info->max_rank = P.max_rank;
    info->n_static_steps = P.n_static_steps;
    info->flops_ma = P.flops_ma;
    info->flops_sa = P.flops_sa;
    info->flops_exec = P.flops_exec;
    info->bytes_min = P.bytes_min;
    info->workspace_bytes = P.ws_bytes;
    info->peak_tensor_bytes = P.peak_tensor_bytes;
    int64_t up = 0;
    for (const auto &u : P.uploads) up += (int64_t)u.second.size();
    info->upload_bytes = up;
    const PlanObj *po = reinterpret_cast<const PlanObj *>(plan);
    double steps_run = 0;
    for (const tnp::Step &st : P.steps) steps_run += (!po->chain_fused(st.chain) || st.chain_last) ? st.runs : 0.0;
    info->launches_per_call = (int64_t)steps_run + 2 * P.n_batches;  // + leaf fill and accumulate per batch
    info->n_open = (int32_t)P.open_qubits.size();
    info->n_chains = (int32_t)P.chains.size();
    info->amps_per_row = int64_t(1) << P.open_qubits.size();
    return TN_OK;
}

int tn_plan_widths(tn_plan_t plan, int64_t *width_out, int32_t *rank, int32_t *n_slice_vars) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_widths: null plan");
    const tnp::Plan &P = reinterpret_cast<PlanObj *>(plan)->P;
    for (size_t v = 0; v < P.nodes.size(); ++v) {
        if (width_out) width_out[v] = P.nodes[v].n_out;
        if (rank) rank[v] = P.nodes[v].rank;
        if (n_slice_vars) n_slice_vars[v] = (int32_t)P.nodes[v].slices.size();
    }
    return TN_OK;
}

int tn_plan_steps(tn_plan_t plan, tn_step_info *out, int32_t n) {
    if (!plan || (n > 0 && !out)) return set_err(TN_EINVAL, "tn_plan_steps: null argument");
    const tnp::Plan &P = reinterpret_cast<PlanObj *>(plan)->P;
    for (int32_t s = 0; s < n && s < (int32_t)P.steps.size(); ++s) {
        const tnp::Step &st = P.steps[s];
        tn_step_info &r = out[s];
        r.node = st.node;
        r.a = st.a;
        r.b = st.b;
        r.mb = st.mb;
        r.kb = st.kb;
        r.nb = st.nb;
        r.rank_a = P.nodes[st.a].rank;
        r.rank_b = P.nodes[st.b].rank;
        r.level = st.level;
        r.kernel = st.kernel;
        r.n_inst = P.nodes[st.node].n_inst;
        r.n_inst_a = P.nodes[st.a].n_inst;
        r.n_inst_b = P.nodes[st.b].n_inst;
        r.flops = st.flops;
        r.bytes = st.bytes;
        r.runs = st.runs;
        auto run = [](const std::vector<int8_t> &pos) {
            int j = 0;
            while (j < (int)pos.size() && pos[j] == j) ++j;
            return j;
        };
        r.a_run_m = run(st.pAm);
        r.a_run_k = run(st.pAk);
        r.b_run_k = run(st.pBk);
        r.b_run_n = run(st.pBn);
        r.n_groups = st.n_groups;
        r.chain = st.chain;
        r.chain_last = st.chain_last ? 1 : 0;
        for (int j = 0; j < 40; ++j) r.c_pos_m[j] = j < st.mb ? st.pCm[j] : -1;
        for (int j = 0; j < 24; ++j) r.c_pos_n[j] = j < st.nb ? st.pCn[j] : -1;
        int64_t mg = 0;
        for (int64_t g = 0; g < st.n_groups; ++g) mg = std::max(mg, st.group_first[g + 1] - st.group_first[g]);
        r.max_group = mg;
        r.n_pair_tiles = st.n_pair_tiles;
    }
    return TN_OK;
}

int tn_plan_batch_slices(tn_plan_t plan, int64_t batch, int64_t *slice_ids, int64_t n) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_batch_slices: null plan");
    const tnp::Plan &P = reinterpret_cast<PlanObj *>(plan)->P;
    const int64_t per = int64_t(1) << P.m_low;
    if (batch < 0 || batch >= P.n_batches) return set_err(TN_EINVAL, "tn_plan_batch_slices: batch outside [0, n_batches)");
    if (n < per || !slice_ids)
        return set_err(TN_EINVAL, "tn_plan_batch_slices: need room for " + std::to_string(per) + " slice ids");
    for (int64_t sigma = 0; sigma < per; ++sigma) {
        const int64_t v = batch * per + sigma;  // internal slice index
        int64_t ext = 0;
        for (size_t t = 0; t < P.perm.size(); ++t) ext |= ((v >> t) & 1) << P.perm[t];
        slice_ids[sigma] = ext;
    }
    return TN_OK;
}

int tn_plan_bind(tn_plan_t plan, void *workspace, size_t bytes, void *stream) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_bind: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return set_err(TN_EINVAL, "tn_plan_bind: workspace must be a 256-byte aligned device pointer");
    if ((int64_t)bytes < o->P.ws_bytes)
        return set_err(TN_ENOMEM, "tn_plan_bind: workspace has " + std::to_string(bytes) + " bytes, plan needs " +
                                      std::to_string(o->P.ws_bytes));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CU(tnk::init_kernels());
    CU(tnk::init_chain_kernel());
    CU(tnk::init_simt_kernels());
    o->drop_graphs();
    o->ws = static_cast<uint8_t *>(workspace);
    o->ws_bytes = bytes;
    for (auto &u : o->P.uploads) {
        if (u.second.empty()) continue;
        CU(cudaMemcpyAsync(o->ws + u.first, u.second.data(), u.second.size(), cudaMemcpyHostToDevice, st));
    }
    o->err_flag = at<int32_t>(o, o->P.off_scratch);
    CU(cudaMemsetAsync(o->err_flag, 0, 4, st));
    CU(cudaStreamSynchronize(st));
    build_descs(o);
    g_err.clear();
    return TN_OK;
}

int tn_contract(tn_plan_t plan, int precision, int64_t batch_lo, int64_t batch_hi, double *amps, void *stream) {
    if (!plan) return set_err(TN_EINVAL, "tn_contract: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    if (!o->ws) return set_err(TN_ESTATE, "tn_contract: no workspace bound (call tn_plan_bind)");
    if (precision < TN_FP32 || precision > TN_BF16X3) return set_err(TN_EINVAL, "tn_contract: bad precision");
    tnp::Plan &P = o->P;
    if (batch_lo < 0 || batch_hi > P.n_batches || batch_lo > batch_hi)
        return set_err(TN_EINVAL, "tn_contract: batch range outside [0, n_batches)");
    if (P.k == 0 || batch_lo == batch_hi) return TN_OK;
    if (!amps) return set_err(TN_EINVAL, "tn_contract: null amplitude buffer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const tnp::Node &R = P.nodes[P.root];
    const float2 *root = at<const float2>(o, R.buf.data);
    const int32_t *E = at<const int32_t>(o, R.buf.E);
    const int32_t *uniq = at<const int32_t>(o, P.off_uniq);
    auto enqueue = [&]() {
        return run_batches(o, precision, batch_lo, batch_hi, st, [&](int64_t) -> int {
            cudaError_t e = tnk::launch_accumulate(root, E, uniq, P.k, R.n_sig, R.n_out, R.rank, amps, st);
            if (e != cudaSuccess) return set_err(TN_ECUDA, std::string("accumulate: ") + cudaGetErrorString(e));
            return TN_OK;
        });
    };
    if (!P.opt.graphs || o->profile) {
        if (int rc = enqueue()) return rc;
        g_err.clear();
        return TN_OK;
    }
    const PlanObj::GraphKey key{precision, batch_lo, batch_hi, amps};
    auto it = o->graphs.find(key);
    if (it == o->graphs.end()) {
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); nothing runs during capture
        if (!o->cap_stream) CU(cudaStreamCreateWithFlags(&o->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaStream_t user = st;
        st = o->cap_stream;
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue();
        const cudaError_t ec = cudaStreamEndCapture(st, &g);
        st = user;
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return set_err(TN_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ec));
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return set_err(TN_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
        it = o->graphs.emplace(key, ex).first;
    }
    CU(cudaGraphLaunch(it->second, st));
    g_err.clear();
    return TN_OK;
}

int tn_contract_slices(tn_plan_t plan, int precision, const int64_t *slice_ids, int32_t ns, double *partials,
                       void *stream) {
    if (!plan) return set_err(TN_EINVAL, "tn_contract_slices: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    if (!o->ws) return set_err(TN_ESTATE, "tn_contract_slices: no workspace bound");
    if (precision < TN_FP32 || precision > TN_BF16X3) return set_err(TN_EINVAL, "bad precision");
    if (ns < 0 || (ns > 0 && (!slice_ids || !partials))) return set_err(TN_EINVAL, "tn_contract_slices: bad args");
    tnp::Plan &P = o->P;
    const int64_t n_slices = int64_t(1) << P.sliced.size();
    const int64_t per = int64_t(1) << P.m_low;
    std::map<int64_t, std::vector<int32_t>> by_batch;
    std::vector<int64_t> internal(ns);
    for (int32_t i = 0; i < ns; ++i) {
        if (slice_ids[i] < 0 || slice_ids[i] >= n_slices) return set_err(TN_EINVAL, "slice id out of range");
        int64_t v = 0;  // external bit j = P.perm[t]  ->  internal bit t
        for (size_t t = 0; t < P.perm.size(); ++t) v |= ((slice_ids[i] >> P.perm[t]) & 1) << t;
        internal[i] = v;
        by_batch[v / per].push_back(i);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const tnp::Node &R = P.nodes[P.root];
    const float2 *root = at<const float2>(o, R.buf.data);
    const int32_t *E = at<const int32_t>(o, R.buf.E);
    const int32_t *uniq = at<const int32_t>(o, P.off_uniq);
    for (auto &kv : by_batch) {
        const int64_t b = kv.first;
        int rc = run_batches(o, precision, b, b + 1, st, [&](int64_t) -> int {
            for (int32_t i : kv.second) {
                const int64_t sigma = internal[i] % per;
                cudaError_t e = tnk::launch_extract(root, E, uniq, P.k, sigma, R.n_out, R.rank,
                                                    partials + (2 * P.k * i << R.rank), st);
                if (e != cudaSuccess) return set_err(TN_ECUDA, std::string("extract: ") + cudaGetErrorString(e));
            }
            return TN_OK;
        });
        if (rc) return rc;
    }
    g_err.clear();
    return TN_OK;
}

int tn_xeb(const double *amps, int64_t k, int32_t n_qubits, double *xeb_dev, void *stream) {
    if (!amps || !xeb_dev || k <= 0 || n_qubits < 1 || n_qubits > 1000)
        return set_err(TN_EINVAL, "tn_xeb: need k > 0, amplitudes and an output word");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = tnk::launch_xeb(amps, k, std::ldexp(1.0, n_qubits) / double(k), xeb_dev, st);
    if (e != cudaSuccess) return set_err(TN_ECUDA, std::string("xeb: ") + cudaGetErrorString(e));
    g_err.clear();
    return TN_OK;
}

int tn_sample_completions(const double *amps, int64_t k, int32_t n_open, const double *uniform, int64_t *picks,
                          void *stream) {
    if (!amps || !uniform || !picks || k <= 0) return set_err(TN_EINVAL, "tn_sample_completions: need k > 0 and buffers");
    if (n_open < 0 || n_open > TN_MAX_OPEN) return set_err(TN_EINVAL, "tn_sample_completions: n_open outside [0, TN_MAX_OPEN]");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = tnk::launch_sample(amps, k, n_open, uniform, picks, st);
    if (e != cudaSuccess) return set_err(TN_ECUDA, std::string("sample: ") + cudaGetErrorString(e));
    g_err.clear();
    return TN_OK;
}

int tn_pt_moments(const double *amps, int64_t k, int32_t n_qubits, double fidelity, double *out_dev, void *stream) {
    if (!amps || !out_dev || k <= 0 || n_qubits < 1 || n_qubits > 1000)
        return set_err(TN_EINVAL, "tn_pt_moments: need k > 0, amplitudes and 5 output words");
    if (!(fidelity >= 0.0 && fidelity < 1.0)) return set_err(TN_EINVAL, "tn_pt_moments: fidelity outside [0, 1)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = tnk::launch_pt_moments(amps, k, std::ldexp(1.0, n_qubits), fidelity, out_dev, st);
    if (e != cudaSuccess) return set_err(TN_ECUDA, std::string("pt_moments: ") + cudaGetErrorString(e));
    g_err.clear();
    return TN_OK;
}

int tn_pt_histogram(const double *amps, int64_t k, int32_t n_qubits, double x_max, int32_t nbins,
                    uint64_t *counts_dev, void *stream) {
    if (!amps || !counts_dev || k <= 0 || n_qubits < 1 || n_qubits > 1000)
        return set_err(TN_EINVAL, "tn_pt_histogram: need k > 0, amplitudes and a count array");
    if (nbins < 1 || nbins > TN_PT_MAX_BINS || !(x_max > 0.0))
        return set_err(TN_EINVAL, "tn_pt_histogram: need 1 <= nbins <= TN_PT_MAX_BINS and x_max > 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = tnk::launch_pt_hist(amps, k, std::ldexp(1.0, n_qubits), x_max, nbins,
                                        reinterpret_cast<unsigned long long *>(counts_dev), st);
    if (e != cudaSuccess) return set_err(TN_ECUDA, std::string("pt_histogram: ") + cudaGetErrorString(e));
    g_err.clear();
    return TN_OK;
}

int tn_fma_probe(int64_t blocks, int64_t iters, float *out_dev, void *stream) {
    if (blocks <= 0 || blocks > 0x7fffffffLL || iters < 0 || !out_dev)
        return set_err(TN_EINVAL, "tn_fma_probe: need 0 < blocks < 2^31, iters >= 0 and an output buffer");
    CU(tnk::launch_fma_probe(blocks, iters, out_dev, reinterpret_cast<cudaStream_t>(stream)));
    g_err.clear();
    return TN_OK;
}

int tn_contract_static(tn_plan_t plan, int precision, double *amps, void *stream) {
    if (!plan) return set_err(TN_EINVAL, "tn_contract_static: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    if (o->P.ws_bytes > (int64_t)TN_STATIC_SCRATCH_BYTES)
        return set_err(TN_ENOMEM, "tn_contract_static: plan needs " + std::to_string(o->P.ws_bytes) +
                                      " workspace bytes; the fixed scratch holds " +
                                      std::to_string((long long)TN_STATIC_SCRATCH_BYTES));
    void *scratch = nullptr;
    if (int rc = static_scratch_address(&scratch)) return rc;
    // bind to the fixed scratch, run every batch, restore the caller's binding
    uint8_t *prev_ws = o->ws;
    const size_t prev_bytes = o->ws_bytes;
    int32_t *prev_flag = o->err_flag;
    const int32_t prev_graphs = o->P.opt.graphs;
    // graphs captured for the caller's own binding stay valid once it is
    // restored: keep them out of the re-bind's reach
    std::map<PlanObj::GraphKey, cudaGraphExec_t> kept;
    kept.swap(o->graphs);
    o->P.opt.graphs = 0;  // every call re-uploads the tables: nothing to replay
    int rc = tn_plan_bind(plan, scratch, (size_t)TN_STATIC_SCRATCH_BYTES, stream);
    if (rc == TN_OK) rc = tn_contract(plan, precision, 0, o->P.n_batches, amps, stream);
    if (rc == TN_OK) rc = tn_plan_check(plan, stream);
    const std::string msg = g_err;
    o->P.opt.graphs = prev_graphs;
    o->ws = prev_ws;
    o->ws_bytes = prev_bytes;
    o->err_flag = prev_flag;
    if (prev_ws) build_descs(o);
    else {
        o->desc.clear();
        o->amap.clear();
    }
    o->drop_graphs();  // none are captured while graphs are off; kept for symmetry
    o->graphs.swap(kept);
    g_err = msg;
    return rc;
}

int tn_plan_set_kernel(tn_plan_t plan, int32_t step, int32_t kernel) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_set_kernel: null plan");
    if (kernel < -1 || kernel > 1) return set_err(TN_EINVAL, "tn_plan_set_kernel: bad kernel family");
    return tn_plan_set_config(plan, step, kernel < 0 ? -1 : 2 * kernel);
}

int tn_plan_set_config(tn_plan_t plan, int32_t step, int32_t config) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_set_config: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    const tnp::Plan &P = o->P;
    if (step < 0 || step >= (int32_t)P.steps.size()) return set_err(TN_EINVAL, "tn_plan_set_config: bad step");
    if (config < -1 || config >= TN_NCONFIG) return set_err(TN_EINVAL, "tn_plan_set_config: bad configuration");
    if (config >= 0 && !config_allowed(P.steps[step], config))
        return set_err(TN_EINVAL, "tn_plan_set_config: per-row kernel needs N <= 16 and K*N <= 256");
    o->config_override.resize(P.steps.size(), -1);
    o->config_override[step] = config;
    o->drop_graphs();
    return TN_OK;
}

int tn_plan_set_chain(tn_plan_t plan, int32_t chain, int32_t enable) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_set_chain: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    if (chain < 0 || chain >= (int32_t)o->P.chains.size()) return set_err(TN_EINVAL, "tn_plan_set_chain: bad chain");
    o->chain_on.resize(o->P.chains.size(), 1);
    o->chain_on[chain] = enable ? 1 : 0;
    o->drop_graphs();
    return TN_OK;
}

int tn_plan_get_chains(tn_plan_t plan, int32_t *enabled, int32_t n) {
    if (!plan || (n > 0 && !enabled)) return set_err(TN_EINVAL, "tn_plan_get_chains: null argument");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    for (int32_t c = 0; c < n && c < (int32_t)o->P.chains.size(); ++c) enabled[c] = o->chain_fused(c) ? 1 : 0;
    return TN_OK;
}

int tn_plan_set_tc_resident_b(tn_plan_t plan, int32_t enable) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_set_tc_resident_b: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    o->tc_resident_b = enable != 0;
    o->drop_graphs();
    return TN_OK;
}

int tn_plan_set_tc_pairs(tn_plan_t plan, int32_t enable) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_set_tc_pairs: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    o->tc_pair = enable != 0;
    o->drop_graphs();
    return TN_OK;
}

int tn_plan_get_configs(tn_plan_t plan, int32_t *config, int32_t n) {
    if (!plan || (n > 0 && !config)) return set_err(TN_EINVAL, "tn_plan_get_configs: null argument");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    for (int32_t s = 0; s < n && s < (int32_t)o->P.steps.size(); ++s) config[s] = effective_config(o, s);
    return TN_OK;
}

int tn_plan_features(tn_plan_t plan, int precision, int32_t config, float *feat, int32_t *eligible, int32_t n) {
    if (!plan || (n > 0 && !feat)) return set_err(TN_EINVAL, "tn_plan_features: null argument");
    if (precision < TN_FP32 || precision > TN_BF16X3) return set_err(TN_EINVAL, "tn_plan_features: bad precision");
    if (config < 0 || config >= TN_NCONFIG) return set_err(TN_EINVAL, "tn_plan_features: bad configuration");
    const tnp::Plan &P = reinterpret_cast<PlanObj *>(plan)->P;
    for (int32_t s = 0; s < n && s < (int32_t)P.steps.size(); ++s) {
        step_features(P, s, precision, config, feat + int64_t(s) * TN_NFEAT);
        if (eligible) eligible[s] = config_allowed(P.steps[s], config) ? 1 : 0;
    }
    return TN_OK;
}

int tn_plan_autotune(tn_plan_t plan, int precision, int32_t reps, const uint8_t *step_mask, double *amps_scratch,
                     double *times, void *stream) {
    if (!plan || !amps_scratch) return set_err(TN_EINVAL, "tn_plan_autotune: null argument");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    if (!o->ws) return set_err(TN_ESTATE, "tn_plan_autotune: no workspace bound");
    if (precision < TN_FP32 || precision > TN_BF16X3) return set_err(TN_EINVAL, "tn_plan_autotune: bad precision");
    if (reps < 1) return set_err(TN_EINVAL, "tn_plan_autotune: reps must be >= 1");
    const tnp::Plan &P = o->P;
    const int ns = (int)P.steps.size();
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int32_t> cur(ns);
    for (int s = 0; s < ns; ++s) cur[s] = effective_config(o, s);
    std::vector<double> best(size_t(ns) * TN_NCONFIG, NAN), ms(ns);
    const bool prof = o->profile;
    o->profile = true;  // CUDA events around every step launch
    o->config_override.assign(ns, -1);
    const int nchains = (int)P.chains.size();
    const std::vector<uint8_t> prev_chain = o->chain_on;
    o->chain_on.assign(nchains, 0);  // configurations are timed on the separate steps
    int rc = TN_OK;
    for (int c = 0; c < TN_NCONFIG && rc == TN_OK; ++c) {
        bool any = false;
        for (int s = 0; s < ns; ++s) {
            const bool sel = (!step_mask || step_mask[s]) && config_allowed(P.steps[s], c);
            o->config_override[s] = sel ? c : cur[s];
            any = any || sel;
        }
        if (!any) continue;
        for (int r = 0; r <= reps && rc == TN_OK; ++r) {
            // the first slice batch of a call runs every step exactly once
            rc = tn_contract(plan, precision, 0, P.n_batches > 0 ? 1 : 0, amps_scratch, stream);
            if (rc == TN_OK) rc = tn_plan_step_times(plan, ms.data(), nullptr, ns);
            if (rc != TN_OK || r == 0) continue;  // the first run warms up
            for (int s = 0; s < ns; ++s) {
                if (o->config_override[s] != c || (step_mask && !step_mask[s])) continue;
                const double t = ms[s];
                double &b = best[size_t(s) * TN_NCONFIG + c];
                if (std::isnan(b) || t < b) b = t;
            }
        }
    }
    if (rc == TN_OK) rc = tn_plan_check(plan, stream);
    o->profile = prof;
    std::string msg = g_err;
    for (int s = 0; s < ns; ++s) {
        int pick = cur[s];
        if (rc == TN_OK && (!step_mask || step_mask[s])) {
            double bt = NAN;
            for (int c = 0; c < TN_NCONFIG; ++c) {
                const double t = best[size_t(s) * TN_NCONFIG + c];
                if (!std::isnan(t) && (std::isnan(bt) || t < bt)) {
                    bt = t;
                    pick = c;
                }
            }
        }
        o->config_override[s] = pick;
    }
    // fused chains: each kept fused only where its kernel beats the sum of
    // its steps' best times (the chain's time is booked on its last step)
    // (with a step mask only some steps were timed: the chains keep their
    // previous setting)
    if (rc != TN_OK || step_mask) o->chain_on = prev_chain;
    if (rc == TN_OK && nchains > 0 && !step_mask) {
        std::vector<double> unfused(nchains, 0.0), fused(nchains, NAN);
        for (int s = 0; s < ns; ++s) {
            const int c = P.steps[s].chain;
            if (c < 0) continue;
            double bt = NAN;
            for (int k = 0; k < TN_NCONFIG; ++k) {
                const double t = best[size_t(s) * TN_NCONFIG + k];
                if (!std::isnan(t) && (std::isnan(bt) || t < bt)) bt = t;
            }
            unfused[c] += std::isnan(bt) ? 0.0 : bt;
        }
        o->chain_on.assign(nchains, 1);
        o->profile = true;
        for (int r = 0; r <= reps && rc == TN_OK; ++r) {
            rc = tn_contract(plan, precision, 0, P.n_batches > 0 ? 1 : 0, amps_scratch, stream);
            if (rc == TN_OK) rc = tn_plan_step_times(plan, ms.data(), nullptr, ns);
            if (rc != TN_OK || r == 0) continue;
            for (int s = 0; s < ns; ++s) {
                const tnp::Step &S = P.steps[s];
                if (S.chain < 0 || !S.chain_last) continue;
                if (std::isnan(fused[S.chain]) || ms[s] < fused[S.chain]) fused[S.chain] = ms[s];
            }
        }
        if (rc == TN_OK) rc = tn_plan_check(plan, stream);
        if (rc != TN_OK) msg = g_err;
        o->profile = prof;
        for (int c = 0; c < nchains; ++c) o->chain_on[c] = (!std::isnan(fused[c]) && fused[c] < unfused[c]) ? 1 : 0;
        if (rc != TN_OK) o->chain_on = prev_chain;
    }
    o->drop_graphs();
    if (times) std::copy(best.begin(), best.end(), times);
    g_err = rc == TN_OK ? std::string() : msg;
    return rc;
}

int tn_plan_select(tn_plan_t plan, int precision, const uint16_t *params16, float margin, void *scratch,
                   size_t scratch_bytes, int32_t *uncertain, void *stream) {
    if (!plan || !params16 || !scratch) return set_err(TN_EINVAL, "tn_plan_select: null argument");
    if (precision < TN_FP32 || precision > TN_BF16X3) return set_err(TN_EINVAL, "tn_plan_select: bad precision");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    const tnp::Plan &P = o->P;
    const int ns = (int)P.steps.size();
    const int64_t rows = int64_t(ns) * TN_NCONFIG;
    const size_t need = size_t(rows) * (TN_NFEAT + 1) * sizeof(float);
    if (scratch_bytes < need)
        return set_err(TN_ENOMEM, "tn_plan_select: scratch needs " + std::to_string(need) + " bytes");
    std::vector<float> X(size_t(rows) * TN_NFEAT), y(rows);
    for (int s = 0; s < ns; ++s)
        for (int c = 0; c < TN_NCONFIG; ++c) step_features(P, s, precision, c, &X[(size_t(s) * TN_NCONFIG + c) * TN_NFEAT]);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float *dX = static_cast<float *>(scratch), *dy = dX + rows * TN_NFEAT;
    CU(cudaMemcpyAsync(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    CU(tnk::mlp_forward_f16(params16, dX, rows, dy, st));
    CU(cudaMemcpyAsync(y.data(), dy, y.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    o->config_override.resize(ns, -1);
    for (int s = 0; s < ns; ++s) {
        int b1 = -1;
        float y1 = 0.f, y2 = 0.f;
        bool have2 = false;
        for (int c = 0; c < TN_NCONFIG; ++c) {
            if (!config_allowed(P.steps[s], c)) continue;
            const float v = y[size_t(s) * TN_NCONFIG + c];
            if (b1 < 0 || v < y1) {
                if (b1 >= 0) {
                    y2 = y1;
                    have2 = true;
                }
                y1 = v;
                b1 = c;
            } else if (!have2 || v < y2) {
                y2 = v;
                have2 = true;
            }
        }
        o->config_override[s] = b1;
        if (uncertain) uncertain[s] = (have2 && y2 - y1 < margin) ? 1 : 0;
    }
    o->drop_graphs();
    g_err.clear();
    return TN_OK;
}

size_t tn_mlp_grad_scratch_bytes(int64_t n) { return tnk::mlp_grad_scratch_bytes(n); }

int tn_mlp_forward(const float *params, const float *X, int64_t n, float *y, void *stream) {
    if (!params || n < 0 || (n > 0 && (!X || !y))) return set_err(TN_EINVAL, "tn_mlp_forward: bad arguments");
    CU(tnk::mlp_forward(params, X, n, y, reinterpret_cast<cudaStream_t>(stream)));
    return TN_OK;
}

int tn_mlp_grad(const float *params, const float *X, const float *t, int64_t n, float *grad, float *loss,
                void *scratch, size_t scratch_bytes, void *stream) {
    if (!params || !X || !t || !grad || !scratch || n <= 0) return set_err(TN_EINVAL, "tn_mlp_grad: bad arguments");
    if (scratch_bytes < tnk::mlp_grad_scratch_bytes(n))
        return set_err(TN_ENOMEM, "tn_mlp_grad: scratch needs " + std::to_string(tnk::mlp_grad_scratch_bytes(n)) +
                                      " bytes");
    CU(tnk::mlp_grad(params, X, t, n, grad, loss, static_cast<float *>(scratch), reinterpret_cast<cudaStream_t>(stream)));
    return TN_OK;
}

int tn_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr, float beta1,
                float beta2, float eps, void *stream) {
    if (!params || !grad || !m || !v || step < 1) return set_err(TN_EINVAL, "tn_mlp_adam: bad arguments");
    CU(tnk::mlp_adam(params, grad, m, v, step, lr, beta1, beta2, eps, reinterpret_cast<cudaStream_t>(stream)));
    return TN_OK;
}

int tn_mlp_to_half(const float *params, uint16_t *params16, void *stream) {
    if (!params || !params16) return set_err(TN_EINVAL, "tn_mlp_to_half: null argument");
    CU(tnk::mlp_to_half(params, params16, reinterpret_cast<cudaStream_t>(stream)));
    return TN_OK;
}

int tn_mlp_forward_f16(const uint16_t *params16, const float *X, int64_t n, float *y, void *stream) {
    if (!params16 || n < 0 || (n > 0 && (!X || !y))) return set_err(TN_EINVAL, "tn_mlp_forward_f16: bad arguments");
    CU(tnk::mlp_forward_f16(params16, X, n, y, reinterpret_cast<cudaStream_t>(stream)));
    return TN_OK;
}

int tn_plan_check(tn_plan_t plan, void *stream) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_check: null plan");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    if (!o->ws) return TN_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t flag = 0;
    CU(cudaMemcpyAsync(&flag, o->err_flag, 4, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (flag) {
        CU(cudaMemsetAsync(o->err_flag, 0, 4, st));
        CU(cudaStreamSynchronize(st));
        return set_err(TN_ETIMEOUT, "a bounded device-side wait gave up (tensor-core pipeline)");
    }
    return TN_OK;
}

int tn_plan_profile(tn_plan_t plan, int enable) {
    if (!plan) return set_err(TN_EINVAL, "tn_plan_profile: null plan");
    reinterpret_cast<PlanObj *>(plan)->profile = enable != 0;
    return TN_OK;
}

int tn_plan_step_times(tn_plan_t plan, double *ms, int32_t *kernel, int32_t n) {
    if (!plan || !ms) return set_err(TN_EINVAL, "tn_plan_step_times: null argument");
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    for (int32_t i = 0; i < n; ++i) {
        ms[i] = 0.0;
        if (kernel) kernel[i] = i < (int32_t)o->step_kernel.size() ? o->step_kernel[i] : -1;
    }
    for (size_t q = 0; q < o->ev_used; ++q) {
        CU(cudaEventSynchronize(o->ev[2 * q + 1]));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, o->ev[2 * q], o->ev[2 * q + 1]));
        if (o->ev_step[q] < n) ms[o->ev_step[q]] += t;
    }
    return TN_OK;
}

void tn_destroy(tn_plan_t plan) {
    if (!plan) return;
    PlanObj *o = reinterpret_cast<PlanObj *>(plan);
    o->drop_graphs();
    if (o->cap_stream) cudaStreamDestroy(o->cap_stream);
    for (cudaEvent_t e : o->ev) cudaEventDestroy(e);
    delete o;
}

}  // extern "C"
