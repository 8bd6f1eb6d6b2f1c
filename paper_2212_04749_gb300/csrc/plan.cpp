// Host planner: fused network, reuse-instance DAG, step schedule, workspace.
// See plan.hpp for the overview.  No CUDA here: tn_plan runs on any host.
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <string>
#include <unordered_map>

extern "C" void tn_options_default(tn_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->workspace_limit = int64_t(64) << 30;
    opt->slice_batch_log2 = -1;
    opt->rescale = 1;
    opt->fuse = 0;
    opt->fuse_max_bits = 7;
    opt->graphs = 1;
}

namespace tnp {

namespace {

using M2 = std::array<cd, 4>;  // row-major 2x2

M2 eye2() { return {cd(1), cd(0), cd(0), cd(1)}; }

M2 mul2(const M2 &a, const M2 &b) {
    M2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) c[2 * i + j] = a[2 * i] * b[j] + a[2 * i + 1] * b[2 + j];
    return c;
}

M2 gate2(const tn_gate &g) {
    M2 m;
    for (int i = 0; i < 4; ++i) m[i] = cd(g.m[2 * i], g.m[2 * i + 1]);
    return m;
}

// First-fit allocator over byte offsets, 256-byte granules.
struct Arena {
    int64_t base = 0, top = 0, high = 0;
    std::map<int64_t, int64_t> free_;  // offset -> size
    static int64_t align(int64_t x) { return (x + 255) & ~int64_t(255); }
    int64_t alloc(int64_t bytes) {
        bytes = align(std::max<int64_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                int64_t off = it->first, sz = it->second;
                free_.erase(it);
                if (sz > bytes) free_[off + bytes] = sz - bytes;
                return off;
            }
        }
        int64_t off = top;
        top += bytes;
        high = std::max(high, top);
        return off;
    }
    void release(int64_t off, int64_t bytes) {
        bytes = align(std::max<int64_t>(bytes, 1));
        auto it = free_.emplace(off, bytes).first;
        // coalesce with next
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
                it = pv;
            }
        }
        if (it->first + it->second == top) {
            top = it->first;
            free_.erase(it);
        }
    }
};

template <class T>
void push_upload(Plan &p, int64_t off, const std::vector<T> &v) {
    std::vector<uint8_t> bytes(v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(bytes.data(), v.data(), bytes.size());
    p.uploads.emplace_back(off, std::move(bytes));
}

}  // namespace

bool build_network(const tn_circuit *circ, Network &net, std::string &err) {
    if (!circ || circ->n_qubits < 1 || circ->n_qubits > 64 || circ->n_gates < 0 ||
        (circ->n_gates > 0 && !circ->gates)) {
        err = "invalid circuit header (need 1 <= n_qubits <= 64)";
        return false;
    }
    const int n = circ->n_qubits;
    net = Network();
    net.n_qubits = n;
    std::vector<M2> pend(n, eye2());
    std::vector<int> last(n, -1);
    std::vector<std::array<cd, 16>> G;  // raw 4x4 gate per tensor
    std::vector<std::array<M2, 2>> U;   // absorbed input-side products
    for (int gi = 0; gi < circ->n_gates; ++gi) {
        const tn_gate &g = circ->gates[gi];
        if (g.q1 < 0) {
            if (g.q0 < 0 || g.q0 >= n) {
                err = "gate " + std::to_string(gi) + ": qubit out of range";
                return false;
            }
            pend[g.q0] = mul2(gate2(g), pend[g.q0]);
            continue;
        }
        if (g.q0 < 0 || g.q1 >= n || g.q0 >= g.q1) {
            err = "gate " + std::to_string(gi) + ": two-qubit gate needs 0 <= q0 < q1 < n";
            return false;
        }
        const int t = (int)net.leaves.size();
        LeafTensor L{};
        L.gate = gi;
        L.qa = g.q0;
        L.qb = g.q1;
        std::array<cd, 16> gm;
        for (int i = 0; i < 16; ++i) gm[i] = cd(g.m[2 * i], g.m[2 * i + 1]);
        std::array<M2, 2> u;
        const int qs[2] = {g.q0, g.q1};
        for (int s = 0; s < 2; ++s) {
            const int q = qs[s];
            if (last[q] >= 0) {
                const int e = net.n_edges++;
                net.edge_ends.push_back({last[q], t});
                LeafTensor &P = net.leaves[last[q]];
                const int slot = (P.qa == q) ? 0 : 1;
                P.legs[slot] = Leg{LEG_BOND, e};
                L.legs[2 + s] = Leg{LEG_BOND, e};
            } else {
                L.legs[2 + s] = Leg{LEG_FIXED, -1};
            }
            L.legs[s] = Leg{LEG_OUT, q};
            u[s] = pend[q];
            pend[q] = eye2();
            last[q] = t;
        }
        net.leaves.push_back(L);
        G.push_back(gm);
        U.push_back(u);
    }
    for (int q = 0; q < n; ++q) {
        if (last[q] < 0) {
            err = "qubit " + std::to_string(q) + " takes part in no two-qubit gate";
            return false;
        }
    }
    net.n_tensors = (int)net.leaves.size();
    net.out_tensor = last;
    // entries: T[oa,ob,ia,ib] = sum V_a[oa,x] V_b[ob,y] G[2x+y, 2z+w] U_a[z,ia] U_b[w,ib]
    for (int t = 0; t < net.n_tensors; ++t) {
        LeafTensor &L = net.leaves[t];
        M2 V[2];
        for (int s = 0; s < 2; ++s) {
            const int q = s == 0 ? L.qa : L.qb;
            V[s] = (L.legs[s].kind == LEG_OUT) ? pend[q] : eye2();
        }
        for (int oa = 0; oa < 2; ++oa)
            for (int ob = 0; ob < 2; ++ob)
                for (int ia = 0; ia < 2; ++ia)
                    for (int ib = 0; ib < 2; ++ib) {
                        cd acc = 0;
                        if ((L.legs[2].kind != LEG_FIXED || ia == 0) &&
                            (L.legs[3].kind != LEG_FIXED || ib == 0)) {
                            for (int x = 0; x < 2; ++x)
                                for (int y = 0; y < 2; ++y)
                                    for (int z = 0; z < 2; ++z)
                                        for (int w = 0; w < 2; ++w)
                                            acc += V[0][2 * oa + x] * V[1][2 * ob + y] *
                                                   G[t][4 * (2 * x + y) + (2 * z + w)] *
                                                   U[t][0][2 * z + ia] * U[t][1][2 * w + ib];
                        }
                        L.t[((oa * 2 + ob) * 2 + ia) * 2 + ib] = acc;
                    }
    }
    return true;
}

namespace {

struct Builder {
    Plan &P;
    std::string &err;
    int &code;
    int T = 0, NN = 0, m = 0;
    std::vector<std::vector<int32_t>> oi;  // node -> per distinct bitstring out-instance
    std::vector<int> slice_of;             // bond edge -> internal slice index (-1: not sliced)
    bool bad_offsets = false;              // set by layout_workspace's self-check
    std::vector<std::vector<int>> low_bits; // per node: bonds its consumer contracts (edge-id order)
    std::vector<std::vector<int>> tails;    // per node: its other bonds, in its consumer's row/column order

    bool fail(int c, const std::string &msg) {
        code = c;
        err = msg;
        return false;
    }

    // Reuse-instance DAG over the distinct bitstrings (SM Sec. III): the
    // out-instances of a node are the distinct projections of the
    // bitstrings onto its output qubits, ordered by (A-child instance,
    // B-child instance) so that instances sharing their A operand are
    // adjacent (one wide GEMM per shared A).
    void out_instances() {
        const int64_t ku = P.k_unique;
        oi.assign(NN, {});
        // leaves: the values of their (at most a few) output qubits
        std::vector<int32_t> key(ku);
        for (int v = 0; v < T; ++v) {
            Node &nd = P.nodes[v];
            const int no = (int)nd.outs.size();
            for (int64_t u = 0; u < ku; ++u) {
                int val = 0;
                for (int t = 0; t < no; ++t) val |= int(P.ubits[u][nd.outs[t]]) << t;
                key[u] = val;
            }
            std::vector<int32_t> id(size_t(1) << no, -1);
            for (int64_t u = 0; u < ku; ++u) id[key[u]] = 0;
            std::vector<int32_t> vals;
            for (int32_t x = 0; x < int32_t(id.size()); ++x)
                if (id[x] >= 0) {
                    id[x] = (int32_t)vals.size();
                    vals.push_back(x);
                }
            if (vals.empty()) vals.push_back(0);
            nd.leaf_outval = vals;
            nd.n_out = (int)vals.size();
            oi[v].resize(ku);
            for (int64_t u = 0; u < ku; ++u) oi[v][u] = ku > 0 ? id[key[u]] : 0;
        }
        // internal nodes: the distinct (A instance, B instance) pairs of the
        // bitstrings, in that order -- two counting-sort passes (by B, then
        // stably by A) instead of a comparison sort per node
        std::vector<int32_t> ord(ku), tmp(ku), cnt;
        for (int v = T; v < NN; ++v) {
            Node &nd = P.nodes[v];
            // major key: the operand the step reads as A (the larger one)
            const bool left_big = a_is_left(P.nodes[nd.left], P.nodes[nd.right]);
            const int a = left_big ? nd.left : nd.right, b = left_big ? nd.right : nd.left;
            const int32_t na = P.nodes[a].n_out, nb = P.nodes[b].n_out;
            const std::vector<int32_t> &ka = oi[a], &kb = oi[b];
            std::vector<int32_t> &oa = left_big ? nd.outL : nd.outR, &ob = left_big ? nd.outR : nd.outL;
            oa.clear();
            ob.clear();
            oi[v].resize(ku);
            if (int64_t(na) * nb <= (int64_t(1) << 16)) {
                // few possible pairs: a table over all of them, scanned in
                // (A, B) order
                const int32_t np = na * nb;
                cnt.assign(size_t(np), -1);
                for (int64_t u = 0; u < ku; ++u) cnt[size_t(ka[u]) * nb + kb[u]] = 0;
                for (int32_t x = 0; x < np; ++x)
                    if (cnt[x] == 0) {
                        cnt[x] = (int32_t)oa.size();
                        oa.push_back(x / nb);
                        ob.push_back(x % nb);
                    }
                for (int64_t u = 0; u < ku; ++u) oi[v][u] = cnt[size_t(ka[u]) * nb + kb[u]];
                if (oa.empty()) {
                    oa.push_back(0);
                    ob.push_back(0);
                }
                nd.n_out = (int)oa.size();
                continue;
            }
            auto pass = [&](const std::vector<int32_t> &k, int32_t nk, const std::vector<int32_t> &in,
                            std::vector<int32_t> &out) {
                cnt.assign(size_t(nk) + 1, 0);
                for (int64_t i = 0; i < ku; ++i) ++cnt[k[in[i]] + 1];
                for (int32_t x = 0; x < nk; ++x) cnt[x + 1] += cnt[x];
                for (int64_t i = 0; i < ku; ++i) out[cnt[k[in[i]]]++] = in[i];
            };
            std::iota(tmp.begin(), tmp.end(), 0);
            pass(kb, nb, tmp, ord);
            pass(ka, na, ord, tmp);  // tmp: u sorted by (A, B), ties in input order
            int32_t pa = -1, pb = -1;
            for (int64_t i = 0; i < ku; ++i) {
                const int32_t u = tmp[i];
                if (ka[u] != pa || kb[u] != pb) {
                    pa = ka[u];
                    pb = kb[u];
                    oa.push_back(pa);
                    ob.push_back(pb);
                }
                oi[v][u] = int32_t(oa.size()) - 1;
            }
            if (oa.empty()) {
                oa.push_back(0);
                ob.push_back(0);
            }
            nd.n_out = (int)oa.size();
        }
    }

    // The operand a step streams as A: the one likely to hold more entries
    // over its bitstring instances, so that B -- read by every group -- is
    // the smaller.  The estimate, rank + min(output qubits below, 16), does
    // not depend on the bitstrings, so a bitstring alone and the same
    // bitstring in a batch run their steps with the same operand roles (the
    // reuse-invariance of an instance's arithmetic); ties by rank, then the
    // left child.
    static bool a_is_left(const Node &l, const Node &r) {
        const int sl = l.rank + std::min<int>((int)l.outs.size(), 16);
        const int sr = r.rank + std::min<int>((int)r.outs.size(), 16);
        if (sl != sr) return sl > sr;
        return l.rank >= r.rank;
    }

    static std::vector<int32_t> compress_map(const std::vector<int> &parent_low,
                                             const std::vector<int> &child_low) {
        // sigma over parent_low bits -> sigma over child_low bits (a subset)
        std::vector<int> pos;
        for (int j : child_low) pos.push_back(int(std::find(parent_low.begin(), parent_low.end(), j) -
                                                  parent_low.begin()));
        const int64_t n = int64_t(1) << parent_low.size();
        std::vector<int32_t> out(n);
        for (int64_t s = 0; s < n; ++s) {
            int32_t c = 0;
            for (size_t t = 0; t < pos.size(); ++t) c |= int32_t((s >> pos[t]) & 1) << t;
            out[s] = c;
        }
        return out;
    }

    bool schedule(int m_low) {
        P.m_low = m_low;
        const int h = m - m_low;
        P.n_batches = int64_t(1) << h;
        for (int v = 0; v < NN; ++v) {
            Node &nd = P.nodes[v];
            nd.slices_low.clear();
            nd.hmask = 0;
            for (int t : nd.slices) {
                if (t < m_low) nd.slices_low.push_back(t);
                else nd.hmask |= uint64_t(1) << (t - m_low);
            }
            nd.level = nd.hmask ? __builtin_ctzll(nd.hmask) : 64;
            nd.n_sig = int64_t(1) << nd.slices_low.size();
            nd.n_inst = nd.n_sig * nd.n_out;
            nd.buf = NodeBuf();
            nd.step = -1;
            nd.last_use = -1;
        }
        for (int v = T; v < NN; ++v) {
            Node &nd = P.nodes[v];
            nd.sigL = compress_map(nd.slices_low, P.nodes[nd.left].slices_low);
            nd.sigR = compress_map(nd.slices_low, P.nodes[nd.right].slices_low);
        }
        // A node is kept across slice batches when its parent is recomputed
        // more often than it is (the parent depends on a sliced edge it does
        // not): the slice analogue of storing the tensor before a branching
        // node of the reuse tree (SM Sec. III.C).
        for (int v = 0; v < NN; ++v) {
            Node &nd = P.nodes[v];
            nd.persistent = (v < T) || (nd.parent >= 0 && nd.level > P.nodes[nd.parent].level);
        }
        // steps in SSA order
        P.steps.clear();
        P.n_static_steps = 0;
        for (int v = T; v < NN; ++v) {
            Node &nd = P.nodes[v];
            Step st;
            st.node = v;
            const Node &l = P.nodes[nd.left], &r = P.nodes[nd.right];
            const bool left_big = a_is_left(l, r);
            st.a = left_big ? nd.left : nd.right;
            st.b = left_big ? nd.right : nd.left;
            st.level = nd.level;
            nd.step = (int)P.steps.size();
            P.n_static_steps += nd.level == 64;
            P.steps.push_back(st);
        }
        // Layouts.  Every node is stored with the bonds its consumer contracts
        // (L = its open bonds shared with its sibling, in edge-id order) as
        // the lowest address bits, so that both operands of every step are
        // K-major with the same k order; the producing step's epilogue writes
        // that layout directly.  Leaves got theirs in make_plan.
        P.max_rank = 0;
        for (int v = 0; v < T; ++v) P.max_rank = std::max(P.max_rank, P.nodes[v].rank);
        for (Step &st : P.steps) {
            Node &nd = P.nodes[st.node];
            const Node &A = P.nodes[st.a], &B = P.nodes[st.b];
            auto in = [](const std::vector<int> &v, int e) { return std::find(v.begin(), v.end(), e) != v.end(); };
            // rows: A's bits above K in address order; columns: B's likewise.
            // Both start with the bits that the next step contracts (the
            // lowest bits of C), so consecutive rows store to neighbouring
            // addresses.
            std::vector<int> kk, mord, nord;
            for (int e : A.layout) (in(B.layout, e) ? kk : mord).push_back(e);
            for (int e : B.layout)
                if (!in(A.layout, e)) nord.push_back(e);
            nd.layout = low_bits[st.node];
            nd.layout.insert(nd.layout.end(), tails[st.node].begin(), tails[st.node].end());
            auto pos = [](const std::vector<int> &lay, int e) {
                return int8_t(std::find(lay.begin(), lay.end(), e) - lay.begin());
            };
            st.mb = (int)mord.size();
            st.kb = (int)kk.size();
            st.nb = (int)nord.size();
            st.pAm.clear(); st.pAk.clear(); st.pBk.clear(); st.pBn.clear(); st.pCm.clear(); st.pCn.clear();
            for (int e : mord) { st.pAm.push_back(pos(A.layout, e)); st.pCm.push_back(pos(nd.layout, e)); }
            for (int e : kk) { st.pAk.push_back(pos(A.layout, e)); st.pBk.push_back(pos(B.layout, e)); }
            for (int e : nord) { st.pBn.push_back(pos(B.layout, e)); st.pCn.push_back(pos(nd.layout, e)); }
            nd.rank = (int)nd.layout.size();
            for (int j = 0; j < st.kb; ++j)
                if (st.pAk[j] != j || st.pBk[j] != j)
                    return fail(TN_EUNSUPPORTED, "internal error: operand not K-major");
            for (int j = 0; j < st.mb; ++j)
                if (st.pAm[j] != st.kb + j || st.pCm[j] >= (int)nd.layout.size())
                    return fail(TN_EUNSUPPORTED, "internal error: A operand not row-affine");
            for (int j = 0; j < st.nb; ++j)
                if (st.pBn[j] != st.kb + j || st.pCn[j] >= (int)nd.layout.size())
                    return fail(TN_EUNSUPPORTED, "internal error: B operand not column-affine");
            if ((int)nd.layout.size() != st.mb + st.nb)
                return fail(TN_EUNSUPPORTED, "internal error: output layout");
            P.max_rank = std::max(P.max_rank, nd.rank);
            if (nd.rank > 40 || st.mb > 40 || st.kb > 24 || st.nb > 24)
                return fail(TN_EUNSUPPORTED, "intermediate rank above 40 (or contracted/free bits above 24)");
            const double macs = std::ldexp(1.0, st.mb + st.kb + st.nb);
            st.flops = 8.0 * double(nd.n_inst) * macs;
            st.bytes = 8.0 * (double(A.n_inst) * std::ldexp(1.0, A.rank) +
                              double(B.n_inst) * std::ldexp(1.0, B.rank) +
                              double(nd.n_inst) * std::ldexp(1.0, nd.rank));
            st.runs = st.level >= h ? 1.0 : std::ldexp(1.0, h - st.level);
            // groups: runs of consecutive output instances reading one A instance
            const bool a_left = st.a == nd.left;
            const std::vector<int32_t> &sgA = a_left ? nd.sigL : nd.sigR;
            const std::vector<int32_t> &otA = a_left ? nd.outL : nd.outR;
            st.group_first.clear();
            int64_t prev = -1;
            for (int64_t i = 0; i < nd.n_inst; ++i) {
                const int64_t sg = i / nd.n_out, bt = i % nd.n_out;
                const int64_t ai = int64_t(sgA[sg]) * A.n_out + otA[bt];
                if (ai != prev) st.group_first.push_back(i);
                prev = ai;
            }
            st.group_first.push_back(nd.n_inst);
            st.n_groups = (int64_t)st.group_first.size() - 1;
            // GEMM column tiles of 64 complex columns over each group's
            // concatenated instances (N columns each)
            st.col_tiles.clear();
            for (int64_t g = 0; g < st.n_groups; ++g) {
                const int64_t cols = (st.group_first[g + 1] - st.group_first[g]) << st.nb;
                for (int64_t t = 0; t * 64 < cols; ++t) st.col_tiles.push_back((g << 20) | t);
            }
            // kernel family: the per-row kernel takes a small B (N <= 16,
            // K*N <= 256) when few instances share an A (under 16 columns per
            // A on average); everything else is a GEMM over instance groups
            const double cols_per_a = std::ldexp(double(nd.n_inst) / double(st.n_groups), st.nb);
            st.kernel = (st.nb <= 4 && st.kb + st.nb <= 8 && cols_per_a < 16.0) ? 0 : 1;
        }
        for (int s = 0; s < (int)P.steps.size(); ++s) {
            P.nodes[P.steps[s].a].last_use = s;
            P.nodes[P.steps[s].b].last_use = s;
        }
        return true;
    }

    // (A instance, B instance) of output instance i of step st
    std::pair<int32_t, int32_t> inst_ab(const Step &st, int64_t i) const {
        const Node &nd = P.nodes[st.node];
        const bool a_left = st.a == nd.left;
        const std::vector<int32_t> &sgA = a_left ? nd.sigL : nd.sigR, &otA = a_left ? nd.outL : nd.outR;
        const std::vector<int32_t> &sgB = a_left ? nd.sigR : nd.sigL, &otB = a_left ? nd.outR : nd.outL;
        const int64_t sg = i / nd.n_out, bt = i % nd.n_out;
        return {int32_t(int64_t(sgA[sg]) * P.nodes[st.a].n_out + otA[bt]),
                int32_t(int64_t(sgB[sg]) * P.nodes[st.b].n_out + otB[bt])};
    }

    // Bit maps of a candidate chain (see Chain); false if a tile exceeds
    // 2^dt entries.
    bool chain_bits(const std::vector<int> &ch, int dt, Chain &c) const {
        const int L = (int)ch.size();
        const Step &s1 = P.steps[ch[0]];
        const Node &A1 = P.nodes[s1.a];
        c = Chain();
        // follow every free bit of A_1 through the chain; the ones no step
        // contracts are the outside bits
        std::vector<std::vector<int>> opos;  // per outside bit: its address bit in C_1 .. C_L
        for (int i = 0; i < s1.mb; ++i) {
            int idx = i;
            bool alive = true;
            std::vector<int> at;
            for (int j = 0; j < L && alive; ++j) {
                const int p = P.steps[ch[j]].pCm[idx];
                at.push_back(p);
                if (j + 1 < L) {
                    const int kn = P.steps[ch[j + 1]].kb;
                    if (p < kn) alive = false;
                    else idx = p - kn;
                }
            }
            if (!alive) continue;
            c.o_in_pos.push_back(int8_t(s1.kb + i));
            c.o_out_pos.push_back(int8_t(at.back()));
            opos.push_back(at);
        }
        // widen the tiles: the lowest outside bits (by address in A_1) join
        // every tile as pass-through rows, until the largest tile reaches
        // 2^dt entries, so that a warp has enough rows to spread over lanes
        {
            int widest = A1.rank - (int)opos.size();
            for (int j = 0; j < L; ++j)
                widest = std::max(widest, P.nodes[P.steps[ch[j]].node].rank - (int)opos.size());
            if (widest > dt) return false;
            int extra = std::min(dt - widest, (int)opos.size());
            while (extra-- > 0) {
                size_t lo = 0;
                for (size_t q = 1; q < opos.size(); ++q)
                    if (c.o_in_pos[q] < c.o_in_pos[lo]) lo = q;
                opos.erase(opos.begin() + lo);
                c.o_in_pos.erase(c.o_in_pos.begin() + lo);
                c.o_out_pos.erase(c.o_out_pos.begin() + lo);
            }
        }
        c.no = (int)opos.size();
        if (c.no > 40) return false;
        std::vector<int> prev;  // tile bits (address bits, ascending) of the current A operand
        for (int p = 0; p < A1.rank; ++p)
            if (std::find(c.o_in_pos.begin(), c.o_in_pos.end(), p) == c.o_in_pos.end()) prev.push_back(p);
        c.tin = (int)prev.size();
        if (c.tin > dt) return false;
        for (int p : prev) c.in_pos.push_back(int8_t(p));
        for (int j = 0; j < L; ++j) {
            const Step &st = P.steps[ch[j]];
            const int rank = P.nodes[st.node].rank;
            std::vector<int> cur;
            for (int p = 0; p < rank; ++p) {
                bool outside = false;
                for (const auto &at : opos) outside = outside || at[j] == p;
                if (!outside) cur.push_back(p);
            }
            if ((int)cur.size() > dt) return false;
            std::vector<int8_t> code;
            for (int p : cur) {
                int8_t v = -1;
                for (int i = 0; i < st.nb; ++i)
                    if (st.pCn[i] == p) v = int8_t(0x80 | i);
                for (int i = 0; i < st.mb && v == -1; ++i)
                    if (st.pCm[i] == p) {
                        const int pa = st.kb + i;  // address bit in A
                        const auto it = std::find(prev.begin(), prev.end(), pa);
                        if (it == prev.end()) return false;  // cannot happen: non-outside m bits are tile bits
                        v = int8_t(it - prev.begin());
                    }
                if (v == -1) return false;
                code.push_back(v);
            }
            // the contracted bits are the lowest tile bits of A
            for (int k = 0; k < st.kb; ++k)
                if (k >= (int)prev.size() || prev[k] != k) return false;
            c.tbits.push_back((int)cur.size());
            c.code.push_back(code);
            prev = cur;
        }
        for (int p : prev) c.out_pos.push_back(int8_t(p));
        // index tables
        c.inoff.assign(size_t(1) << c.tin, 0);
        for (size_t e = 0; e < c.inoff.size(); ++e)
            for (int b = 0; b < c.tin; ++b)
                if ((e >> b) & 1) c.inoff[e] += int64_t(1) << c.in_pos[b];
        c.outoff.assign(size_t(1) << c.tbits.back(), 0);
        for (size_t t = 0; t < c.outoff.size(); ++t)
            for (size_t b = 0; b < c.out_pos.size(); ++b)
                if ((t >> b) & 1) c.outoff[t] += int64_t(1) << c.out_pos[b];
        c.rowin.assign(L, {});
        c.rowout.assign(L, {});
        c.colout.assign(L, {});
        for (int j = 0; j < L; ++j) {
            const Step &st = P.steps[ch[j]];
            const int tb = c.tbits[j];
            const int rows = 1 << (tb - st.nb);
            c.rowin[j].assign(rows, 0);
            c.rowout[j].assign(rows, 0);
            for (int r = 0; r < rows; ++r) {
                int qb = 0;
                for (int b = 0; b < tb; ++b) {
                    const int cd = c.code[j][b];
                    if (cd & 0x80) continue;  // n bit
                    if ((r >> qb) & 1) {
                        c.rowin[j][r] |= 1 << cd;
                        c.rowout[j][r] |= 1 << b;
                    }
                    ++qb;
                }
            }
            c.colout[j].assign(size_t(1) << st.nb, 0);
            for (int n = 0; n < (1 << st.nb); ++n)
                for (int b = 0; b < tb; ++b) {
                    const int cd = c.code[j][b];
                    if ((cd & 0x80) && ((n >> (cd & 0x7f)) & 1)) c.colout[j][n] |= 1 << b;
                }
        }
        return true;
    }

    // Fused chains (opt.fuse): greedy, in step order.
    void find_chains() {
        P.chains.clear();
        for (Step &st : P.steps) {
            st.chain = -1;
            st.chain_last = false;
        }
        if (!P.opt.fuse) return;
        const int dt = std::max(1, std::min(P.opt.fuse_max_bits > 0 ? P.opt.fuse_max_bits : 7, CHAIN_MAX_TILE_BITS));
        const int ns = (int)P.steps.size();
        std::vector<int> consumer(P.nodes.size(), -1);
        for (int s = 0; s < ns; ++s) {
            consumer[P.steps[s].a] = s;
            consumer[P.steps[s].b] = s;
        }
        auto small = [](const Step &st) { return st.kb + st.nb <= 8; };
        for (int s = 0; s < ns; ++s) {
            if (P.steps[s].chain >= 0 || !small(P.steps[s])) continue;
            std::vector<int> ch{s};
            Chain c;
            while ((int)ch.size() < CHAIN_MAX_STEPS) {
                const Step &last = P.steps[ch.back()];
                const int nx = consumer[last.node];
                if (nx < 0) break;
                const Step &nst = P.steps[nx];
                if (nst.a != last.node || !small(nst) || nst.level != last.level || nst.chain >= 0) break;
                if (P.nodes[nst.node].n_inst != P.nodes[last.node].n_inst || P.nodes[last.node].persistent) break;
                std::vector<int> trial = ch;
                trial.push_back(nx);
                if (!chain_bits(trial, dt, c)) break;
                ch = trial;
            }
            if (ch.size() < 2) continue;
            chain_bits(ch, dt, c);
            c.steps = ch;
            for (int q : ch) P.steps[q].chain = (int)P.chains.size();
            P.steps[ch.back()].chain_last = true;
            // the chain reads A_1 and every B_j when it runs, at its last
            // step: their buffers must live until then
            P.nodes[P.steps[ch[0]].a].last_use = ch.back();
            for (int q : ch) P.nodes[P.steps[q].b].last_use = ch.back();
            P.chains.push_back(c);
        }
    }

    // Workspace layout; returns total bytes.
    int64_t layout_workspace(bool emit) {
        Plan &p = P;
        if (emit) p.uploads.clear();
        int64_t off = 0;
        auto take = [&](int64_t bytes) {
            int64_t o = off;
            off += Arena::align(std::max<int64_t>(bytes, 1));
            return o;
        };
        // full leaf tensors, extended layout: open bonds, outputs, sliced legs
        std::vector<int64_t> full_off(T);
        int64_t full_elems = 0;
        for (int v = 0; v < T; ++v) {
            const LeafTensor &L = p.net.leaves[v];
            int legs_used = 0;
            for (int g = 0; g < 4; ++g) legs_used += L.legs[g].kind != LEG_FIXED;
            full_off[v] = full_elems;
            full_elems += int64_t(1) << legs_used;
        }
        p.off_leaf_full = take(full_elems * 8);
        // internal slice index of each leaf's sliced legs, increasing
        std::vector<std::vector<int>> leaf_sl(T);
        for (int v = 0; v < T; ++v) {
            const LeafTensor &L = p.net.leaves[v];
            for (int g = 0; g < 4; ++g)
                if (L.legs[g].kind == LEG_BOND && slice_of[L.legs[g].id] >= 0)
                    leaf_sl[v].push_back(slice_of[L.legs[g].id]);
            std::sort(leaf_sl[v].begin(), leaf_sl[v].end());
        }
        if (emit) {
            std::vector<float> full(full_elems * 2, 0.f);
            for (int v = 0; v < T; ++v) {
                const LeafTensor &L = p.net.leaves[v];
                const Node &nd = p.nodes[v];
                int bitpos[4] = {-1, -1, -1, -1};
                for (int g = 0; g < 4; ++g) {
                    if (L.legs[g].kind == LEG_BOND && slice_of[L.legs[g].id] < 0) {
                        auto it = std::find(nd.layout.begin(), nd.layout.end(), L.legs[g].id);
                        bitpos[g] = int(it - nd.layout.begin());
                    }
                }
                int nxt = nd.rank;
                for (int g = 0; g < 4; ++g)
                    if (L.legs[g].kind == LEG_OUT) bitpos[g] = nxt++;
                for (int t : leaf_sl[v])
                    for (int g = 0; g < 4; ++g)
                        if (L.legs[g].kind == LEG_BOND && slice_of[L.legs[g].id] == t) bitpos[g] = nxt++;
                for (int idx = 0; idx < 16; ++idx) {
                    const int bits[4] = {(idx >> 3) & 1, (idx >> 2) & 1, (idx >> 1) & 1, idx & 1};
                    bool ok = true;
                    int64_t e = 0;
                    for (int g = 0; g < 4; ++g) {
                        if (L.legs[g].kind == LEG_FIXED) { ok &= bits[g] == 0; continue; }
                        e |= int64_t(bits[g]) << bitpos[g];
                    }
                    if (!ok) continue;
                    full[2 * (full_off[v] + e)] = (float)L.t[idx].real();
                    full[2 * (full_off[v] + e) + 1] = (float)L.t[idx].imag();
                }
            }
            push_upload(p, p.off_leaf_full, full);
        }
        // max-|x| words ordered by recompute level, so that the words of the
        // nodes recomputed in a batch form one prefix
        std::vector<int> by_level(NN);
        std::iota(by_level.begin(), by_level.end(), 0);
        std::stable_sort(by_level.begin(), by_level.end(),
                         [&](int x, int y) { return p.nodes[x].level < p.nodes[y].level; });
        p.off_emax = off;
        p.emax_prefix.assign(65, 0);
        for (int v : by_level) p.nodes[v].buf.mx = take(p.nodes[v].n_inst * 4);
        p.emax_bytes = off - p.off_emax;
        for (int lv = 0; lv <= 64; ++lv) {
            int64_t end = p.off_emax;
            for (int v : by_level)
                if (p.nodes[v].level <= lv) end = std::max(end, p.nodes[v].buf.mx + Arena::align(p.nodes[v].n_inst * 4));
            p.emax_prefix[lv] = end - p.off_emax;
        }
        for (int v = 0; v < NN; ++v) {
            Node &nd = p.nodes[v];
            nd.buf.E = take(nd.n_inst * 4);
            if (v >= T) {
                nd.buf.sig = take(nd.n_sig * 8);
                nd.buf.out = take(int64_t(nd.n_out) * 8);
                if (emit) {
                    std::vector<int32_t> s(nd.sigL), o(nd.outL);
                    s.insert(s.end(), nd.sigR.begin(), nd.sigR.end());
                    o.insert(o.end(), nd.outR.begin(), nd.outR.end());
                    push_upload(p, nd.buf.sig, s);
                    push_upload(p, nd.buf.out, o);
                }
            } else if (emit) {
                std::vector<int32_t> zeros(nd.n_inst, 0);
                push_upload(p, nd.buf.E, zeros);
            }
            if (nd.persistent) nd.buf.data = take(nd.n_inst * (int64_t(8) << nd.rank));
        }
        // fill jobs (one per leaf instance)
        std::vector<LeafHigh> highs;
        std::vector<FillJob> jobs;
        for (int v = 0; v < T; ++v) {
            const Node &nd = p.nodes[v];
            LeafHigh hh{};
            const std::vector<int> &sj = leaf_sl[v];
            const int base_bit = nd.rank + (int)nd.outs.size();
            for (size_t t = 0; t < sj.size(); ++t) {
                if (sj[t] >= p.m_low) {
                    hh.j[hh.cnt] = sj[t] - p.m_low;
                    hh.stride[hh.cnt] = int32_t(1) << (base_bit + int(t));
                    hh.cnt++;
                }
            }
            const int32_t hidx = (int32_t)highs.size();
            highs.push_back(hh);
            for (int64_t sg = 0; sg < nd.n_sig; ++sg) {
                int64_t slice_bits = 0;  // bit t <-> sj[t]; low ones from sigma
                for (size_t t = 0; t < sj.size(); ++t) {
                    auto it = std::find(nd.slices_low.begin(), nd.slices_low.end(), sj[t]);
                    if (it != nd.slices_low.end())
                        slice_bits |= ((sg >> int(it - nd.slices_low.begin())) & 1) << t;
                }
                for (int b = 0; b < nd.n_out; ++b) {
                    FillJob j{};
                    const int64_t inst = sg * nd.n_out + b;
                    j.dst = (nd.buf.data / 8) + inst * (int64_t(1) << nd.rank);
                    const int64_t block = (slice_bits << nd.outs.size()) | nd.leaf_outval[b];
                    j.src = (p.off_leaf_full / 8) + full_off[v] + (block << nd.rank);
                    j.leaf_high = hidx;
                    j.n = int32_t(1) << nd.rank;
                    jobs.push_back(j);
                }
            }
        }
        // every fill job copies inside its leaf's instance buffer, from inside
        // the full-leaf region, for every value of the looped sliced legs
        for (size_t q = 0; q < jobs.size(); ++q) {
            const FillJob &j = jobs[q];
            const LeafHigh &hh = highs[j.leaf_high];
            int64_t hmax = 0;
            for (int c = 0; c < hh.cnt; ++c) hmax += hh.stride[c];
            if (j.src < p.off_leaf_full / 8 || j.src + hmax + j.n > p.off_leaf_full / 8 + full_elems)
                bad_offsets = true;
        }
        p.n_fill_jobs = (int64_t)jobs.size();
        p.off_fill_jobs = take(int64_t(jobs.size()) * sizeof(FillJob));
        p.off_leaf_high = take(int64_t(highs.size()) * sizeof(LeafHigh));
        if (emit) {
            push_upload(p, p.off_fill_jobs, jobs);
            push_upload(p, p.off_leaf_high, highs);
        }
        p.off_uniq = take(p.k * 4);
        if (emit) {
            std::vector<int32_t> r(p.k);
            for (int64_t i = 0; i < p.k; ++i) r[i] = oi[p.root][p.uniq_of[i]];
            push_upload(p, p.off_uniq, r);
        }
        p.off_scratch = take(256);
        for (Step &st : p.steps) {
            st.off_groups = take(int64_t(st.group_first.size()) * 8);
            if (emit) push_upload(p, st.off_groups, st.group_first);
            st.off_col_tiles = take(int64_t(st.col_tiles.size()) * 8);
            if (emit) push_upload(p, st.off_col_tiles, st.col_tiles);
            // one 16-byte record per column tile and one int32 pair per
            // output instance, so that a kernel reaches every index it needs
            // with a single load instead of a chain of dependent ones
            const Node &nd = p.nodes[st.node];
            const bool a_left = st.a == nd.left;
            const std::vector<int32_t> &sgA = a_left ? nd.sigL : nd.sigR, &otA = a_left ? nd.outL : nd.outR;
            const std::vector<int32_t> &sgB = a_left ? nd.sigR : nd.sigL, &otB = a_left ? nd.outR : nd.outL;
            const int64_t noA = p.nodes[st.a].n_out, noB = p.nodes[st.b].n_out;
            st.off_tile_rec = take(int64_t(st.col_tiles.size()) * 16);
            st.off_inst_ab = take(nd.n_inst * 8);
            if (emit) {
                std::vector<int32_t> ab(2 * nd.n_inst);
                for (int64_t i = 0; i < nd.n_inst; ++i) {
                    const int64_t sg = i / nd.n_out, bt = i % nd.n_out;
                    ab[2 * i] = int32_t(int64_t(sgA[sg]) * noA + otA[bt]);
                    ab[2 * i + 1] = int32_t(int64_t(sgB[sg]) * noB + otB[bt]);
                }
                std::vector<int32_t> rec(4 * st.col_tiles.size());
                for (size_t t = 0; t < st.col_tiles.size(); ++t) {
                    const int64_t g = st.col_tiles[t] >> 20, ct = st.col_tiles[t] & 0xfffff;
                    const int64_t i0 = st.group_first[g];
                    rec[4 * t] = int32_t(i0);
                    rec[4 * t + 1] = int32_t(st.group_first[g + 1] - i0);
                    rec[4 * t + 2] = ab[2 * i0];
                    rec[4 * t + 3] = int32_t(ct * 64);
                }
                push_upload(p, st.off_inst_ab, ab);
                push_upload(p, st.off_tile_rec, rec);
            }
            st.n_pair_tiles = 0;
            st.off_pair_tab = -1;
            if (st.nb == 6) {
                for (int64_t g = 0; g < st.n_groups; ++g) {
                    const int64_t nct = st.group_first[g + 1] - st.group_first[g];
                    st.n_pair_tiles += nct + (nct & 1);
                }
                st.off_pair_tab = take(st.n_pair_tiles * 8);
                if (emit) {
                    std::vector<int32_t> pt;
                    pt.reserve(size_t(2 * st.n_pair_tiles));
                    int64_t f = 0, fp = 0;
                    for (int64_t g = 0; g < st.n_groups; ++g) {
                        const int64_t nct = st.group_first[g + 1] - st.group_first[g];
                        for (int64_t t = 0; t < nct + (nct & 1); ++t) {
                            pt.push_back(int32_t(f));
                            pt.push_back(int32_t(fp));
                        }
                        f += nct;
                        fp += nct + (nct & 1);
                    }
                    push_upload(p, st.off_pair_tab, pt);
                }
            }
        }
        // room for the packed B operand of the largest step that can take it
        // (N >= 64, K >= 8, 64 <= M < 2^31: every B instance, 16 bytes per
        // complex entry, K padded to chunks of 16); steps run one at a time,
        // so one region serves all; steps above the cap (256 MiB, or 1/16 of
        // the workspace limit if that is more) keep B resident or stream it
        p.bpack_bytes = 0;
        const int64_t bpack_cap = std::max(int64_t(256) << 20, p.opt.workspace_limit / 16);
        for (const Step &st : p.steps) {
            if (st.nb < 6 || st.kb < 3 || st.kb > 24 || st.mb < 6 || st.mb > 30) continue;
            const int64_t nch = ((int64_t(1) << st.kb) + 15) / 16;
            const int64_t bytes = p.nodes[st.b].n_inst * (int64_t(1) << (st.nb - 6)) * nch * 16384;
            if (bytes <= bpack_cap) p.bpack_bytes = std::max(p.bpack_bytes, bytes);
        }
        p.off_bpack = p.bpack_bytes > 0 ? take(p.bpack_bytes) : -1;
        for (Chain &c : p.chains) {
            const Step &last = p.steps[c.steps.back()];
            const int64_t ni = p.nodes[last.node].n_inst;
            const int L = (int)c.steps.size();
            c.off_tab = take(ni * (L + 1) * 4);
            {
                std::vector<uint8_t> blob;
                auto put = [&](const void *src, size_t n) {
                    const uint8_t *b = static_cast<const uint8_t *>(src);
                    blob.insert(blob.end(), b, b + n);
                };
                put(c.inoff.data(), c.inoff.size() * 8);
                put(c.outoff.data(), c.outoff.size() * 8);
                for (int j = 0; j < L; ++j) {
                    put(c.rowin[j].data(), c.rowin[j].size() * 4);
                    put(c.rowout[j].data(), c.rowout[j].size() * 4);
                    put(c.colout[j].data(), c.colout[j].size() * 4);
                }
                c.off_idx = take((int64_t)blob.size());
                if (emit) push_upload(p, c.off_idx, blob);
            }
            if (emit) {
                std::vector<int32_t> tab(size_t(ni) * (L + 1));
                for (int64_t i = 0; i < ni; ++i) {
                    int64_t cur = i;
                    for (int j = L - 1; j >= 0; --j) {
                        const auto ab = inst_ab(p.steps[c.steps[j]], cur);
                        tab[size_t(i) * (L + 1) + 1 + j] = ab.second;
                        cur = ab.first;
                    }
                    tab[size_t(i) * (L + 1)] = int32_t(cur);
                }
                push_upload(p, c.off_tab, tab);
            }
        }
        // transient intermediates: first-fit over one full pass of the steps
        Arena ar;
        ar.base = ar.top = ar.high = off;
        p.peak_tensor_bytes = 0;
        const int nst = (int)p.steps.size();
        for (int s = 0; s < nst; ++s) {
            const Step &st = p.steps[s];
            Node &nd = p.nodes[st.node];
            const int64_t bytes = nd.n_inst * (int64_t(8) << nd.rank);
            if (!nd.persistent) nd.buf.data = ar.alloc(bytes);
            for (int c : {st.a, st.b}) {
                Node &ch = p.nodes[c];
                if (ch.persistent || ch.last_use != s) continue;
                ar.release(ch.buf.data, ch.n_inst * (int64_t(8) << ch.rank));
            }
            p.peak_tensor_bytes = std::max(p.peak_tensor_bytes, bytes);
        }
        const int64_t total = Arena::align(ar.high);
        // every node buffer inside the workspace; every job destination inside its leaf
        for (int v = 0; v < NN; ++v) {
            const Node &nd = p.nodes[v];
            if (nd.buf.data < 0 || nd.buf.data + nd.n_inst * (int64_t(8) << nd.rank) > total) bad_offsets = true;
            if (nd.buf.E < 0 || nd.buf.mx < 0) bad_offsets = true;
        }
        for (const FillJob &j : jobs) {
            bool inside = false;
            for (int v = 0; v < T && !inside; ++v) {
                const Node &nd = p.nodes[v];
                const int64_t b0 = nd.buf.data / 8, b1 = b0 + nd.n_inst * (int64_t(1) << nd.rank);
                inside = j.dst >= b0 && j.dst + j.n <= b1;
            }
            if (!inside) bad_offsets = true;
        }
        return total;
    }
};

}  // namespace

bool make_plan(const tn_circuit *circ, const uint8_t *bits, int64_t k, const int32_t *ssa,
               const int32_t *sliced, int32_t n_sliced, const tn_options *opt, Plan &P,
               std::string &err, int &code) {
    code = TN_EINVAL;
    if (!build_network(circ, P.net, err)) return false;
    const int n = P.net.n_qubits;
    const int T = P.net.n_tensors;
    P.n_qubits = n;
    if (opt) P.opt = *opt;
    else tn_options_default(&P.opt);
    if (P.opt.workspace_limit <= 0) P.opt.workspace_limit = int64_t(64) << 30;
    // Open output qubits (correlated batches): the output leg of each becomes
    // a bond edge with one end.  No step contracts it, so it stays in the
    // index sets up to the root, which then holds 2^|open| amplitudes per
    // instance (the absorbed final single-qubit gates stay in the leaf).
    // The bitstrings' values at open qubits are ignored.
    const int n_edges_closed = P.net.n_edges;
    {
        const uint64_t om = uint64_t(P.opt.open_mask);
        if (n < 64 && (om >> n) != 0) { err = "open_mask: a qubit beyond n_qubits"; return false; }
        P.open_qubits.clear();
        for (int q = 0; q < n; ++q)
            if ((om >> q) & 1u) P.open_qubits.push_back(q);
        if ((int)P.open_qubits.size() > TN_MAX_OPEN) {
            err = "open_mask: more than TN_MAX_OPEN open qubits";
            return false;
        }
        for (int q : P.open_qubits) {
            const int t = P.net.out_tensor[q];
            LeafTensor &L = P.net.leaves[t];
            const int slot = (L.legs[0].kind == LEG_OUT && L.legs[0].id == q) ? 0 : 1;
            const int e = P.net.n_edges++;
            P.net.edge_ends.push_back({t, -1});
            L.legs[slot] = Leg{LEG_BOND, e};
        }
    }
    if (k < 0 || (k > 0 && !bits)) { err = "bitstrings: need k >= 0 and a buffer"; return false; }
    if (k > (int64_t(1) << 30)) { err = "bitstrings: k too large"; return false; }
    // distinct bitstrings (c6: deduplicate, answer per input row)
    P.k = k;
    P.uniq_of.assign(k, 0);
    {
        std::unordered_map<std::string, int32_t> seen;
        for (int64_t r = 0; r < k; ++r) {
            std::string key(reinterpret_cast<const char *>(bits + r * n), n);
            for (int q = 0; q < n; ++q)
                if (uint8_t(key[q]) > 1) { err = "bitstrings: entries must be 0 or 1"; return false; }
            for (int q : P.open_qubits) key[q] = 0;
            auto it = seen.find(key);
            if (it == seen.end()) {
                it = seen.emplace(key, (int32_t)P.ubits.size()).first;
                P.ubits.emplace_back(key.begin(), key.end());
            }
            P.uniq_of[r] = it->second;
        }
        P.k_unique = (int64_t)P.ubits.size();
    }
    // sliced edges
    if (n_sliced < 0 || n_sliced > 40 || (n_sliced > 0 && !sliced)) { err = "sliced edges: bad count"; return false; }
    P.sliced.assign(sliced, sliced + n_sliced);
    {
        std::set<int> s(P.sliced.begin(), P.sliced.end());
        if ((int)s.size() != n_sliced) { err = "sliced edges: duplicates"; return false; }
        for (int e : P.sliced)
            if (e < 0 || e >= n_edges_closed) { err = "sliced edges: id out of range"; return false; }
    }
    // tree
    const int NN = 2 * T - 1;
    P.nodes.assign(NN, Node());
    if (T > 1 && !ssa) { err = "tree: missing"; return false; }
    {
        std::vector<int> used(NN, 0);
        for (int i = 0; i < T - 1; ++i) {
            const int a = ssa[2 * i], b = ssa[2 * i + 1];
            if (a < 0 || b < 0 || a >= T + i || b >= T + i || a == b) {
                err = "tree: pair " + std::to_string(i) + " refers to a node not yet created";
                return false;
            }
            if (++used[a] > 1 || ++used[b] > 1) {
                err = "tree: node used twice (pair " + std::to_string(i) + ")";
                return false;
            }
            P.nodes[T + i].left = a;
            P.nodes[T + i].right = b;
            P.nodes[a].parent = T + i;
            P.nodes[b].parent = T + i;
        }
    }
    P.root = NN - 1;
    // leaves: layout = open (unsliced) bond legs, ib first; outs; slices
    std::vector<int> slice_index(P.net.n_edges, -1);
    for (int j = 0; j < n_sliced; ++j) slice_index[P.sliced[j]] = j;  // external j for now
    for (int v = 0; v < T; ++v) {
        const LeafTensor &L = P.net.leaves[v];
        Node &nd = P.nodes[v];
        for (int g = 3; g >= 0; --g) {
            if (L.legs[g].kind == LEG_BOND) {
                if (slice_index[L.legs[g].id] >= 0) nd.slices.push_back(slice_index[L.legs[g].id]);
                else nd.layout.push_back(L.legs[g].id);
            }
        }
        for (int g = 0; g < 2; ++g)
            if (L.legs[g].kind == LEG_OUT) nd.outs.push_back(L.legs[g].id);
        std::sort(nd.outs.begin(), nd.outs.end());
        std::sort(nd.slices.begin(), nd.slices.end());
        nd.rank = (int)nd.layout.size();
    }
    std::vector<std::vector<int>> open(NN);
    for (int v = 0; v < T; ++v) {
        open[v] = P.nodes[v].layout;
        std::sort(open[v].begin(), open[v].end());
    }
    for (int v = T; v < NN; ++v) {
        Node &nd = P.nodes[v];
        const Node &a = P.nodes[nd.left], &b = P.nodes[nd.right];
        std::set_symmetric_difference(open[nd.left].begin(), open[nd.left].end(), open[nd.right].begin(),
                                      open[nd.right].end(), std::back_inserter(open[v]));
        nd.rank = (int)open[v].size();
        std::set_union(a.outs.begin(), a.outs.end(), b.outs.begin(), b.outs.end(), std::back_inserter(nd.outs));
        std::set_union(a.slices.begin(), a.slices.end(), b.slices.begin(), b.slices.end(),
                       std::back_inserter(nd.slices));
    }
    if ((int)P.nodes[P.root].outs.size() + (int)P.open_qubits.size() != n) {
        err = "tree: root does not hold every output leg";
        return false;
    }
    // bonds each node shares with its sibling (contracted by its consumer)
    std::vector<std::vector<int>> low_bits(NN);
    for (int v = T; v < NN; ++v) {
        const int a = P.nodes[v].left, b = P.nodes[v].right;
        std::vector<int> kset;
        std::set_intersection(open[a].begin(), open[a].end(), open[b].begin(), open[b].end(),
                              std::back_inserter(kset));
        low_bits[a] = kset;
        low_bits[b] = kset;
    }
    // Address order above the contracted bonds: the bonds the grandparent's
    // step contracts first, then the rest, each in edge-id order.  That is
    // the consumer's row (resp. column) order, so every operand is
    // row-affine: address = k + 2^kb * m.
    std::vector<std::vector<int>> tails(NN);
    for (int v = 0; v < NN; ++v) {
        const int p = P.nodes[v].parent;
        auto has = [](const std::vector<int> &s, int e) { return std::binary_search(s.begin(), s.end(), e); };
        std::vector<int> rest;
        for (int e : open[v]) {
            if (has(low_bits[v], e)) continue;
            if (p >= 0 && has(low_bits[p], e)) tails[v].push_back(e);
            else rest.push_back(e);
        }
        tails[v].insert(tails[v].end(), rest.begin(), rest.end());
    }
    // leaf layouts: the contracted bonds first (edge-id order), then the tail
    for (int v = 0; v < T; ++v) {
        Node &nd = P.nodes[v];
        nd.layout = low_bits[v];
        nd.layout.insert(nd.layout.end(), tails[v].begin(), tails[v].end());
    }

    Builder B{P, err, code, 0, 0, 0, {}, {}, false, {}};
    B.T = T;
    B.NN = NN;
    B.m = n_sliced;
    B.low_bits = low_bits;
    B.tails = tails;
    B.out_instances();
    // Internal slice order.  The first m_low sliced edges run side by side in
    // one pass; the rest are looped over, bit t - m_low of the batch index,
    // and in batch b only the nodes whose looped edges include a bit below
    // ctz(b) + 1 are recomputed.  A node with looped edge set S is then
    // computed 2^(h - min S) times instead of 2^|S| (depth-first reuse over
    // slices, ideal when every node's edges are the most significant bits).
    // Candidate orders are scored with that exact count, weighted by each
    // node's flops, and the cheapest is kept.
    {
        std::vector<double> fl(NN, 0.0);
        for (int v = T; v < NN; ++v) {
            const Node &nd = P.nodes[v];
            const int uni = (P.nodes[nd.left].rank + P.nodes[nd.right].rank + nd.rank) / 2;
            fl[v] = 8.0 * std::ldexp(1.0, uni) * nd.n_out;
        }
        auto cost = [&](const std::vector<int> &order) {  // order[t] = external j
            std::vector<int> pos(n_sliced);
            for (int t = 0; t < n_sliced; ++t) pos[order[t]] = t;
            double c = 0;
            for (int v = T; v < NN; ++v) {
                if (P.nodes[v].slices.empty()) { c += fl[v]; continue; }
                int lo = n_sliced;
                for (int j : P.nodes[v].slices) lo = std::min(lo, pos[j]);
                c += fl[v] * std::ldexp(1.0, n_sliced - lo);
            }
            return c;
        };
        std::vector<std::vector<int>> cands;
        std::vector<double> first(n_sliced, 0), nodes_with(n_sliced, 0), flops_with(n_sliced, 0);
        for (int j = 0; j < n_sliced; ++j) {
            const auto &ends = P.net.edge_ends[P.sliced[j]];
            first[j] = std::min(P.nodes[ends[0]].parent, P.nodes[ends[1]].parent);
        }
        for (int v = T; v < NN; ++v)
            for (int j : P.nodes[v].slices) {
                nodes_with[j] += 1;
                flops_with[j] += fl[v];
            }
        for (int c = 0; c < 3; ++c) {
            std::vector<int> ord(n_sliced);
            std::iota(ord.begin(), ord.end(), 0);
            const std::vector<double> &key = c == 0 ? first : (c == 1 ? nodes_with : flops_with);
            // fast-changing (low) bits first: latest met / used by the fewest / cheapest nodes
            std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
                return c == 0 ? key[x] > key[y] : key[x] < key[y];
            });
            cands.push_back(ord);
        }
        size_t best = 0;
        for (size_t c = 1; c < cands.size(); ++c)
            if (cost(cands[c]) < cost(cands[best])) best = c;
        P.perm = cands[best];
        std::vector<int> internal(n_sliced);
        for (int t = 0; t < n_sliced; ++t) internal[P.perm[t]] = t;
        for (Node &nd : P.nodes) {
            for (int &j : nd.slices) j = internal[j];
            std::sort(nd.slices.begin(), nd.slices.end());
        }
        for (int e = 0; e < P.net.n_edges; ++e)
            if (slice_index[e] >= 0) slice_index[e] = internal[slice_index[e]];
    }
    B.slice_of = slice_index;
    // slice batch: explicit, or the largest that fits the workspace limit
    int lo = 0, hi = std::min(n_sliced, 20);
    if (P.opt.slice_batch_log2 >= 0) lo = hi = std::min(P.opt.slice_batch_log2, n_sliced);
    int chosen = -1;
    // Cheap bounds before building a candidate's tables: every instance
    // costs ~48 bytes of host tables (instance maps, group and tile records),
    // and the tensors kept across slice batches (a node whose parent is
    // recomputed more often than it is, and the leaves) plus the largest of
    // the others must fit the workspace together.  Batches that fail either
    // are skipped without being built.
    auto surely_too_big = [&](int ml) {
        std::vector<int> level(NN);
        for (int v = 0; v < NN; ++v) {
            int lv = 64;
            for (int t : P.nodes[v].slices)
                if (t >= ml) lv = std::min(lv, t - ml);
            level[v] = lv;
        }
        double inst = 0.0, kept = 0.0, largest = 0.0;
        for (int v = 0; v < NN; ++v) {
            const Node &nd = P.nodes[v];
            int low = 0;
            for (int t : nd.slices) low += t < ml;
            const double ni = std::ldexp(double(nd.n_out), low);
            const double bytes = ni * std::ldexp(8.0, nd.rank);
            inst += ni;
            if (v < T || (nd.parent >= 0 && level[v] > level[nd.parent])) kept += bytes;
            else largest = std::max(largest, bytes);
        }
        return inst * 48.0 > double(int64_t(8) << 30) || kept + largest > double(P.opt.workspace_limit);
    };
    for (int ml = hi; ml >= lo; --ml) {
        if (ml > lo && surely_too_big(ml)) continue;
        if (!B.schedule(ml)) return false;
        const int64_t ws = B.layout_workspace(false);
        if (ws <= P.opt.workspace_limit || ml == lo) {
            chosen = ml;
            if (ws > P.opt.workspace_limit && P.opt.slice_batch_log2 < 0) {
                code = TN_ENOMEM;
                err = "plan needs " + std::to_string(ws) + " workspace bytes even with one slice per pass";
                return false;
            }
            break;
        }
    }
    // the loop's last schedule() was for `chosen` (layout_workspace(false)
    // only sets offsets that the final layout recomputes)
    B.find_chains();
    for (Node &nd : P.nodes) { nd.buf = NodeBuf(); }
    P.peak_tensor_bytes = 0;
    P.ws_bytes = B.layout_workspace(true);
    if (B.bad_offsets) {
        code = TN_EUNSUPPORTED;
        err = "internal error: workspace layout self-check failed";
        return false;
    }
    // costs
    P.flops_exec = P.flops_ma = P.flops_sa = P.bytes_min = 0;
    for (const Step &st : P.steps) {
        const Node &nd = P.nodes[st.node];
        P.flops_exec += st.flops * st.runs;
        double bytes = st.bytes;
        if (st.chain >= 0) {  // a chain's intermediates are never stored
            const double inner = 8.0 * double(nd.n_inst) * std::ldexp(1.0, nd.rank);
            if (!st.chain_last) bytes -= inner;  // C_j of a non-final step
            if (P.steps[P.chains[st.chain].steps[0]].node != st.node) {
                const Node &A = P.nodes[st.a];
                bytes -= 8.0 * double(A.n_inst) * std::ldexp(1.0, A.rank);  // A_j, j > 1
            }
        }
        P.bytes_min += bytes * st.runs;
        const double macs = std::ldexp(1.0, st.mb + st.kb + st.nb);
        P.flops_ma += 8.0 * macs * std::ldexp(1.0, (int)nd.slices.size()) * nd.n_out;
        P.flops_sa += 8.0 * macs * std::ldexp(1.0, n_sliced) * double(P.k_unique);
    }
    code = TN_OK;
    return true;
}

}  // namespace tnp
