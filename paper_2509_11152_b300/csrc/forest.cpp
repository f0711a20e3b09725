// Descriptor checks and the forest layout of a batch of independent H^2 matrices.
//
// A batch is factorised as one forest: the trees are aligned by height above the
// leaves, so level l of the forest holds the level-(l - (d - d_s)) boxes of every
// tree s of depth d_s.  Each forest level is then processed by one launch per kernel
// and colour for all trees at once (the systems never interact: their near fields,
// fill and Schur targets stay inside one tree).  With one tree the forest numbering is
// the heap numbering of the descriptor.
#include <algorithm>
#include <numeric>

#include "h2rs_internal.h"

namespace h2rs {

static int heap_level(int64_t g) { return 63 - __builtin_clzll((unsigned long long)(g + 1)); }

int HostStructure::level_of(int64_t g) const {
    auto it = std::upper_bound(lev_first.begin(), lev_first.end(), g);
    return (int)(it - lev_first.begin()) - 1;
}

template <class T>
static std::vector<T> host_copy(const T* p, int64_t n, const char* what) {
    H2_REQUIRE(n >= 0, H2_ERR_ARG, std::string("negative length for ") + what);
    H2_REQUIRE(n == 0 || p != nullptr, H2_ERR_ARG, std::string("null array ") + what);
    return std::vector<T>(p, p + n);
}

void read_structure(const h2_matrix_desc* d, HostStructure& H) {
    H2_REQUIRE(d != nullptr, H2_ERR_ARG, "null descriptor");
    H2_REQUIRE(d->n > 0 && d->depth >= 0 && d->depth < 30, H2_ERR_ARG, "bad n or depth");
    H.n = d->n;
    H.d = d->depth;
    H.nnodes = (int64_t(1) << (H.d + 1)) - 1;
    const int64_t nn = H.nnodes, nleaf = int64_t(1) << H.d, first_leaf = nleaf - 1;
    H.node_start = host_copy(d->node_start, nn, "node_start");
    H.node_size = host_copy(d->node_size, nn, "node_size");
    H.rank = host_copy(d->rank, nn, "rank");
    H.U_off = host_copy(d->U_off, nleaf + 1, "U_off");
    H.E_off = host_copy(d->E_off, nn + 1, "E_off");
    H.adm_ptr = host_copy(d->adm_ptr, nn + 1, "adm_ptr");
    H.inad_ptr = host_copy(d->inad_ptr, nn + 1, "inad_ptr");
    H2_REQUIRE(H.adm_ptr[0] == 0 && H.inad_ptr[0] == 0, H2_ERR_ARG, "CSR must start at 0");
    H.adm_col = host_copy(d->adm_col, H.adm_ptr[nn], "adm_col");
    H.S_off = host_copy(d->S_off, H.adm_ptr[nn] + 1, "S_off");
    H.inad_col = host_copy(d->inad_col, H.inad_ptr[nn], "inad_col");
    const int64_t nnear = H.inad_ptr[nn] - H.inad_ptr[first_leaf];
    H.D_off = host_copy(d->D_off, nnear + 1, "D_off");
    H2_REQUIRE(H.node_size[0] == H.n && H.node_start[0] == 0, H2_ERR_ARG, "root must cover 0..n");
    H2_REQUIRE(H.U_off[0] == 0 && H.E_off[0] == 0 && H.S_off[0] == 0 && H.D_off[0] == 0, H2_ERR_ARG,
               "value offsets must start at 0");
    for (int64_t g = 0; g < nn - nleaf; ++g) {
        const int64_t c1 = 2 * g + 1, c2 = 2 * g + 2;
        H2_REQUIRE(H.node_size[c1] + H.node_size[c2] == H.node_size[g] &&
                       H.node_start[c1] == H.node_start[g] &&
                       H.node_start[c2] == H.node_start[g] + H.node_size[c1],
                   H2_ERR_ARG, "children must partition their parent");
    }
    for (int64_t i = 0; i < nleaf; ++i) {
        const int64_t g = first_leaf + i;
        H2_REQUIRE(H.rank[g] >= 0 && H.rank[g] <= H.node_size[g], H2_ERR_ARG, "leaf rank > size");
        H2_REQUIRE(H.U_off[i + 1] - H.U_off[i] == H.node_size[g] * H.rank[g], H2_ERR_ARG, "U_off size");
    }
    for (int64_t g = 1; g < nn; ++g)
        H2_REQUIRE(H.E_off[g + 1] - H.E_off[g] == H.rank[g] * H.rank[(g - 1) / 2], H2_ERR_ARG,
                   "E_off size");
    H2_REQUIRE(H.E_off[1] == 0, H2_ERR_ARG, "the root has no transfer matrix");
    for (int64_t g = 0; g < nn; ++g) {
        const int l = heap_level(g);
        const int64_t lf = (int64_t(1) << l) - 1, ll = (int64_t(1) << (l + 1)) - 1;
        for (int64_t e = H.adm_ptr[g]; e < H.adm_ptr[g + 1]; ++e) {
            const int64_t t = H.adm_col[e];
            H2_REQUIRE(t >= lf && t < ll, H2_ERR_ARG, "admissible pair across levels");
            if (e > H.adm_ptr[g]) H2_REQUIRE(t > H.adm_col[e - 1], H2_ERR_ARG, "adm_col not sorted");
            H2_REQUIRE(H.S_off[e + 1] - H.S_off[e] == H.rank[g] * H.rank[t], H2_ERR_ARG, "S_off size");
        }
        bool self = false;
        for (int64_t e = H.inad_ptr[g]; e < H.inad_ptr[g + 1]; ++e) {
            const int64_t t = H.inad_col[e];
            H2_REQUIRE(t >= lf && t < ll, H2_ERR_ARG, "inadmissible pair across levels");
            self |= t == g;
            if (e > H.inad_ptr[g]) H2_REQUIRE(t > H.inad_col[e - 1], H2_ERR_ARG, "inad_col not sorted");
            if (g >= first_leaf) {
                const int64_t j = e - H.inad_ptr[first_leaf];
                H2_REQUIRE(H.D_off[j + 1] - H.D_off[j] == H.node_size[g] * H.node_size[t], H2_ERR_ARG,
                           "D_off size");
            }
        }
        H2_REQUIRE(self, H2_ERR_ARG, "every node must be in its own near field");
    }
    // the matrix is symmetric, so are both patterns: (g, t) in one => (t, g) in the
    // same one; and no pair is both admissible and inadmissible
    auto has = [](const std::vector<int64_t>& ptr, const std::vector<int64_t>& col, int64_t g, int64_t t) {
        return std::binary_search(col.begin() + ptr[g], col.begin() + ptr[g + 1], t);
    };
    for (int64_t g = 0; g < nn; ++g) {
        for (int64_t e = H.inad_ptr[g]; e < H.inad_ptr[g + 1]; ++e)
            H2_REQUIRE(has(H.inad_ptr, H.inad_col, H.inad_col[e], g), H2_ERR_ARG,
                       "the inadmissible pattern is not symmetric");
        for (int64_t e = H.adm_ptr[g]; e < H.adm_ptr[g + 1]; ++e) {
            H2_REQUIRE(has(H.adm_ptr, H.adm_col, H.adm_col[e], g), H2_ERR_ARG,
                       "the admissible pattern is not symmetric");
            H2_REQUIRE(!has(H.inad_ptr, H.inad_col, g, H.adm_col[e]), H2_ERR_ARG,
                       "a pair is both admissible and inadmissible");
        }
    }
}

// append a chunk, merging it with the previous one when both ranges continue it
static void add_chunk(std::vector<ValueChunk>& v, int sys, int64_t src, int64_t dst, int64_t cnt) {
    if (cnt <= 0) return;
    if (!v.empty()) {
        ValueChunk& b = v.back();
        if (b.sys == sys && b.src + b.cnt == src && b.dst + b.cnt == dst) { b.cnt += cnt; return; }
    }
    v.push_back({sys, src, dst, cnt});
}

void merge_forest(const std::vector<HostStructure>& parts, HostStructure& F, std::vector<int>& order,
                  ForestValues& fv) {
    const int ns = (int)parts.size();
    H2_REQUIRE(ns >= 1, H2_ERR_ARG, "empty batch");
    int D = 0;
    for (const auto& p : parts) D = std::max(D, p.d);
    order.resize(ns);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return parts[a].d > parts[b].d; });
    F = HostStructure{};
    F.d = D;
    F.nsys = ns;
    F.sys_voff.assign(ns + 1, 0);
    for (int s = 0; s < ns; ++s) F.sys_voff[s + 1] = F.sys_voff[s] + parts[s].n;
    F.n = F.sys_voff[ns];
    F.sys_root.resize(ns);
    for (int s = 0; s < ns; ++s) F.sys_root[s] = D - parts[s].d;
    // per level: offset of every present tree, in merged order
    std::vector<std::vector<int64_t>> off(ns, std::vector<int64_t>(D + 1, -1));
    F.lev_cnt.assign(D + 1, 0);
    F.lev_first.assign(D + 1, 0);
    for (int l = 0; l <= D; ++l) {
        int64_t c = 0;
        for (int r = 0; r < ns; ++r) {
            const int s = order[r];
            if (F.sys_root[s] <= l) { off[s][l] = c; c += int64_t(1) << (l - F.sys_root[s]); }
        }
        F.lev_cnt[l] = c;
        if (l > 0) F.lev_first[l] = F.lev_first[l - 1] + F.lev_cnt[l - 1];
    }
    F.nnodes = F.lev_first[D] + F.lev_cnt[D];
    const int64_t nn = F.nnodes, fleaf = F.lev_first[D];
    auto gid = [&](int s, int64_t g) -> int64_t {
        const int ls = heap_level(g);
        const int l = F.sys_root[s] + ls;
        return F.lev_first[l] + off[s][l] + (g - ((int64_t(1) << ls) - 1));
    };
    std::vector<int> src_sys(nn, -1);
    std::vector<int64_t> src_g(nn, -1);
    for (int s = 0; s < ns; ++s)
        for (int64_t g = 0; g < parts[s].nnodes; ++g) {
            const int64_t G = gid(s, g);
            src_sys[G] = s;
            src_g[G] = g;
        }
    F.node_start.resize(nn);
    F.node_size.resize(nn);
    F.rank.resize(nn);
    F.parent.resize(nn);
    F.sys.resize(nn);
    for (int64_t G = 0; G < nn; ++G) {
        const int s = src_sys[G];
        const int64_t g = src_g[G];
        H2_REQUIRE(s >= 0, H2_ERR_ARG, "forest numbering is not a bijection");
        const HostStructure& p = parts[s];
        F.node_start[G] = F.sys_voff[s] + p.node_start[g];
        F.node_size[G] = p.node_size[g];
        F.rank[G] = p.rank[g];
        F.parent[G] = g == 0 ? -1 : gid(s, (g - 1) / 2);
        F.sys[G] = s;
    }
    // leaf bases: one contiguous range of leaves per tree
    const int64_t nleaf = F.lev_cnt[D];
    F.U_off.assign(nleaf + 1, 0);
    for (int64_t i = 0; i < nleaf; ++i) F.U_off[i + 1] = F.U_off[i] + F.node_size[fleaf + i] * F.rank[fleaf + i];
    // transfers, admissible CSR + couplings, inadmissible CSR
    F.E_off.assign(nn + 1, 0);
    F.adm_ptr.assign(nn + 1, 0);
    F.inad_ptr.assign(nn + 1, 0);
    F.S_off.assign(1, 0);
    for (int64_t G = 0; G < nn; ++G) {
        const HostStructure& p = parts[src_sys[G]];
        const int64_t g = src_g[G];
        const int s = src_sys[G];
        F.E_off[G + 1] = F.E_off[G] + (p.E_off[g + 1] - p.E_off[g]);
        for (int64_t e = p.adm_ptr[g]; e < p.adm_ptr[g + 1]; ++e) {
            F.adm_col.push_back(gid(s, p.adm_col[e]));
            F.S_off.push_back(F.S_off.back() + (p.S_off[e + 1] - p.S_off[e]));
        }
        F.adm_ptr[G + 1] = (int64_t)F.adm_col.size();
        for (int64_t e = p.inad_ptr[g]; e < p.inad_ptr[g + 1]; ++e) F.inad_col.push_back(gid(s, p.inad_col[e]));
        F.inad_ptr[G + 1] = (int64_t)F.inad_col.size();
    }
    const int64_t nbase = F.inad_ptr[fleaf];
    F.D_off.assign(F.inad_ptr[nn] - nbase + 1, 0);
    for (int64_t G = fleaf; G < nn; ++G)
        for (int64_t e = F.inad_ptr[G]; e < F.inad_ptr[G + 1]; ++e)
            F.D_off[e - nbase + 1] = F.D_off[e - nbase] + F.node_size[G] * F.node_size[F.inad_col[e]];
    // value chunks (merged order, so that consecutive ranges of one tree coalesce)
    fv = ForestValues{};
    for (int r = 0; r < ns; ++r) {
        const int s = order[r];
        const HostStructure& p = parts[s];
        const int64_t G0 = gid(s, (int64_t(1) << p.d) - 1);
        add_chunk(fv.U, s, 0, F.U_off[G0 - fleaf], p.U_off.back());
        add_chunk(fv.D, s, 0, F.D_off[F.inad_ptr[G0] - nbase], p.D_off.back());
    }
    for (int l = 0; l <= D; ++l)
        for (int r = 0; r < ns; ++r) {
            const int s = order[r];
            if (F.sys_root[s] > l) continue;
            const HostStructure& p = parts[s];
            const int ls = l - F.sys_root[s];
            const int64_t g0 = (int64_t(1) << ls) - 1, g1 = (int64_t(1) << (ls + 1)) - 1;
            const int64_t G0 = gid(s, g0);
            add_chunk(fv.E, s, p.E_off[g0], F.E_off[G0], p.E_off[g1] - p.E_off[g0]);
            add_chunk(fv.S, s, p.S_off[p.adm_ptr[g0]], F.S_off[F.adm_ptr[G0]],
                      p.S_off[p.adm_ptr[g1]] - p.S_off[p.adm_ptr[g0]]);
        }
}

}  // namespace h2rs
