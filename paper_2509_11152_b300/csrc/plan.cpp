// Level planner: integer structure of the strong recursive skeletonisation.
//
// Sec. 2.2: at every level the inadmissible (near-field) blocks form a block-sparse
// graph; a greedy colouring of it gives sets of boxes that can be skeletonised
// concurrently.  Eliminating box i updates every block (j, k) with j, k in N(i)
// (Sec. 2.1 step 3), so the blocks a level can touch are its near field plus the
// "distance two" pairs outside it, plus fill carried from the level below whose
// parent pair is not in the near field (moved to D or kept in F at the level
// close).  Everything here depends only on the block partition, so it is built once
// per matrix; box sizes and ranks are applied per level by the driver.
#include <algorithm>
#include <thread>

#include "h2rs_internal.h"

namespace h2rs {

// f(lo, hi) over [0, n) in contiguous ranges on the host's cores (the plan of a
// million-point matrix walks tens of millions of block pairs)
// (at least `grain` items per thread)
template <class F>
static void parallel_for(int64_t n, F f, int64_t grain = 16) {
    const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nt = std::min<int64_t>(std::min<int64_t>(hw, 32), std::max<int64_t>(1, n / grain));
    if (nt <= 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int64_t t = 1; t < nt; ++t) th.emplace_back(f, n * t / nt, n * (t + 1) / nt);
    f((int64_t)0, n / nt);
    for (auto& x : th) x.join();
}

int LevelStruct::find(int i, int j) const {
    auto b = bcol.begin() + bptr[i];
    auto e = bcol.begin() + bptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    if (it == e || *it != j) return -1;
    return (int)(it - bcol.begin());
}

// near-field CSR of level l (local indices), from A's inadmissible CSR; boxes that are
// not reached at this level (state 0) get empty rows
static void near_graph(const HostStructure& H, int l, LevelStruct& L) {
    L.l = l;
    L.first = H.lev_first[l];
    L.cnt = (int)H.lev_cnt[l];
    L.nb_ptr.assign(L.cnt + 1, 0);
    L.nb_col.clear();
    L.top_boxes.clear();
    L.skel_boxes.clear();
    for (int i = 0; i < L.cnt; ++i) {
        int64_t g = L.first + i;
        if (L.state[i] != 0)
            for (int64_t e = H.inad_ptr[g]; e < H.inad_ptr[g + 1]; ++e)
                L.nb_col.push_back((int)(H.inad_col[e] - L.first));
        std::sort(L.nb_col.begin() + L.nb_ptr[i], L.nb_col.end());
        L.nb_ptr[i + 1] = (int)L.nb_col.size();
        if (L.state[i] == 1) L.skel_boxes.push_back(i);
        if (L.state[i] == 2) L.top_boxes.push_back(i);
    }
}

// first-fit colouring in ascending box index, self loops ignored; only the boxes
// skeletonised at this level are coloured (others keep -1)
static void colour_level(LevelStruct& L) {
    L.colour.assign(L.cnt, -1);
    std::vector<int> mark;
    for (int i : L.skel_boxes) {
        mark.assign(L.nb_ptr[i + 1] - L.nb_ptr[i] + 2, 0);
        for (int e = L.nb_ptr[i]; e < L.nb_ptr[i + 1]; ++e) {
            int j = L.nb_col[e];
            if (j == i) continue;
            int c = L.colour[j];
            if (c >= 0 && c < (int)mark.size()) mark[c] = 1;
        }
        int c = 0;
        while (mark[c]) ++c;
        L.colour[i] = c;
    }
    L.ncolour = L.cnt ? *std::max_element(L.colour.begin(), L.colour.end()) + 1 : 0;
    L.cboxes.assign(L.ncolour, {});
    for (int i : L.skel_boxes) L.cboxes[L.colour[i]].push_back(i);
}

static bool is_near(const LevelStruct& L, int i, int j) {
    auto b = L.nb_col.begin() + L.nb_ptr[i];
    auto e = L.nb_col.begin() + L.nb_ptr[i + 1];
    return std::binary_search(b, e, j);
}

// merged block list = near field U fill pattern (distance-two pairs + carried)
static void block_list(LevelStruct& L, const std::vector<std::pair<int, int>>& carried) {
    // fill of row j: k in N(i) outside N(j), for every eliminated i in N(j) (the near
    // graph is symmetric, so these are the pairs j, k in N(i) of Sec. 2.1 step 3)
    std::vector<std::vector<int>> fill(L.cnt);
    parallel_for(L.cnt, [&](int64_t lo, int64_t hi) {
        for (int j = (int)lo; j < (int)hi; ++j)
            for (int a = L.nb_ptr[j]; a < L.nb_ptr[j + 1]; ++a) {
                const int i = L.nb_col[a];
                if (L.state[i] != 1) continue;        // only eliminated boxes create fill
                for (int b = L.nb_ptr[i]; b < L.nb_ptr[i + 1]; ++b) {
                    const int k = L.nb_col[b];
                    if (!is_near(L, j, k)) fill[j].push_back(k);
                }
            }
    });
    std::vector<std::vector<int>> carr(L.cnt);
    for (auto& pq : carried)
        if (!is_near(L, pq.first, pq.second)) {
            fill[pq.first].push_back(pq.second);
            carr[pq.first].push_back(pq.second);
        }
    // merged rows (near field + fill, columns ascending) and their kinds
    std::vector<std::vector<int>> merged(L.cnt);
    std::vector<std::vector<int8_t>> kinds(L.cnt);
    parallel_for(L.cnt, [&](int64_t lo, int64_t hi) {
        for (int i = (int)lo; i < (int)hi; ++i) {
            auto& f = fill[i];
            std::sort(f.begin(), f.end());
            f.erase(std::unique(f.begin(), f.end()), f.end());
            auto& m = merged[i];
            m.reserve(L.nb_ptr[i + 1] - L.nb_ptr[i] + f.size());
            std::merge(L.nb_col.begin() + L.nb_ptr[i], L.nb_col.begin() + L.nb_ptr[i + 1], f.begin(), f.end(),
                       std::back_inserter(m));
            kinds[i].reserve(m.size());
            for (int j : m) kinds[i].push_back(is_near(L, i, j) ? 0 : 1);
            std::sort(carr[i].begin(), carr[i].end());
        }
    });
    L.bptr.assign(L.cnt + 1, 0);
    for (int i = 0; i < L.cnt; ++i) L.bptr[i + 1] = L.bptr[i] + (int)merged[i].size();
    L.bcol.resize(L.bptr[L.cnt]);
    L.bkind.resize(L.bptr[L.cnt]);
    parallel_for(L.cnt, [&](int64_t lo, int64_t hi) {
        for (int i = (int)lo; i < (int)hi; ++i) {
            std::copy(merged[i].begin(), merged[i].end(), L.bcol.begin() + L.bptr[i]);
            std::copy(kinds[i].begin(), kinds[i].end(), L.bkind.begin() + L.bptr[i]);
        }
    });
    int nb = L.nblocks();
    L.btr.assign(nb, -1);
    L.first_touch.assign(nb, INT_MAX);
    parallel_for(L.cnt, [&](int64_t lo, int64_t hi) {
        for (int i = (int)lo; i < (int)hi; ++i)
            for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b) {
                L.btr[b] = L.find(L.bcol[b], i);
                if (L.bkind[b] == 1 && std::binary_search(carr[i].begin(), carr[i].end(), L.bcol[b]))
                    L.first_touch[b] = -1;
            }
    });
}

// Schur targets per colour (target-owned accumulation) and first touches of fill;
// the colours are listed concurrently, then concatenated in colour order
static void schur_lists(LevelStruct& L) {
    struct Rec { int t, i, a, kpos; };
    struct Part {
        std::vector<int> tblk, tlen, ci, cA, ckpos;
    };
    std::vector<Part> parts(L.ncolour);
    parallel_for(L.ncolour, [&](int64_t lo, int64_t hi) {
        std::vector<Rec> recs;
        for (int c = (int)lo; c < (int)hi; ++c) {
            recs.clear();
            for (int i : L.cboxes[c]) {
                int n0 = L.nb_ptr[i], n1 = L.nb_ptr[i + 1];
                for (int a = n0; a < n1; ++a) {
                    int j = L.nb_col[a];
                    int ablk = L.find(j, i);
                    for (int b = n0; b < n1; ++b) recs.push_back({L.find(j, L.nb_col[b]), i, ablk, b - n0});
                }
            }
            std::sort(recs.begin(), recs.end(), [](const Rec& x, const Rec& y) {
                return x.t != y.t ? x.t < y.t : x.i < y.i;
            });
            Part& P = parts[c];
            for (size_t r = 0; r < recs.size(); ++r) {
                if (r == 0 || recs[r].t != recs[r - 1].t) {
                    P.tblk.push_back(recs[r].t);
                    P.tlen.push_back(0);
                }
                ++P.tlen.back();
                P.ci.push_back(recs[r].i);
                P.cA.push_back(recs[r].a);
                P.ckpos.push_back(recs[r].kpos);
            }
        }
    }, 1);
    L.sch_cptr.assign(1, 0);
    L.sch_tblk.clear();
    L.sch_tptr.assign(1, 0);
    L.sch_ci.clear();
    L.sch_cA.clear();
    L.sch_ckpos.clear();
    for (int c = 0; c < L.ncolour; ++c) {
        const Part& P = parts[c];
        for (size_t q = 0; q < P.tblk.size(); ++q) {
            const int t = P.tblk[q];
            L.sch_tblk.push_back(t);
            L.sch_tptr.push_back(L.sch_tptr.back() + P.tlen[q]);
            if (L.bkind[t] == 1 && L.first_touch[t] == INT_MAX) L.first_touch[t] = c;
        }
        L.sch_ci.insert(L.sch_ci.end(), P.ci.begin(), P.ci.end());
        L.sch_cA.insert(L.sch_cA.end(), P.cA.begin(), P.cA.end());
        L.sch_ckpos.insert(L.sch_ckpos.end(), P.ckpos.begin(), P.ckpos.end());
        L.sch_cptr.push_back((int)L.sch_tblk.size());
    }
}

// block ids per near-field position and forward-solve target lists
static void solve_lists(LevelStruct& L) {
    L.nb_blk.resize(L.nb_col.size());
    L.nb_blkT.resize(L.nb_col.size());
    parallel_for(L.cnt, [&](int64_t lo, int64_t hi) {
        for (int i = (int)lo; i < (int)hi; ++i)
            for (int a = L.nb_ptr[i]; a < L.nb_ptr[i + 1]; ++a) {
                L.nb_blk[a] = L.find(i, L.nb_col[a]);
                L.nb_blkT[a] = L.find(L.nb_col[a], i);
            }
    });
    L.fl_cptr.assign(1, 0);
    L.fl_tbox.clear();
    L.fl_tptr.assign(1, 0);
    L.fl_ci.clear();
    L.fl_cpos.clear();
    struct Rec { int j, i, pos; };
    std::vector<Rec> recs;
    for (int c = 0; c < L.ncolour; ++c) {
        recs.clear();
        for (int i : L.cboxes[c])
            for (int a = L.nb_ptr[i]; a < L.nb_ptr[i + 1]; ++a)
                recs.push_back({L.nb_col[a], i, a - L.nb_ptr[i]});
        std::sort(recs.begin(), recs.end(), [](const Rec& x, const Rec& y) {
            return x.j != y.j ? x.j < y.j : x.i < y.i;
        });
        for (size_t r = 0; r < recs.size(); ++r) {
            if (r == 0 || recs[r].j != recs[r - 1].j) {
                if (r) L.fl_tptr.push_back((int)L.fl_ci.size());
                L.fl_tbox.push_back(recs[r].j);
            }
            L.fl_ci.push_back(recs[r].i);
            L.fl_cpos.push_back(recs[r].pos);
        }
        if (!recs.empty()) L.fl_tptr.push_back((int)L.fl_ci.size());
        L.fl_cptr.push_back((int)L.fl_tbox.size());
    }
}

// structure-only work lists of every colour (first_touch is final after schur_lists)
static void work_lists(LevelStruct& L) {
    L.seg_blk.clear(); L.seg_j.clear(); L.seg_slot.clear();
    L.seg_ptr.assign(1, 0);
    L.seg_cptr.assign(1, 0);
    L.pj_box.clear(); L.pj_blk.clear(); L.pj_blkT.clear();
    L.pj_cptr.assign(1, 0);
    L.zf_box.clear(); L.zf_blk.clear(); L.zf_col.clear();
    L.zn_box.clear(); L.zn_blk.clear(); L.zn_col.clear();
    L.zf_cptr.assign(1, 0);
    L.zn_cptr.assign(1, 0);
    for (int c = 0; c < L.ncolour; ++c) {
        int slot = 0;
        for (int i : L.cboxes[c]) {
            for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b) {
                if (L.bkind[b] != 1 || L.first_touch[b] >= c) continue;
                L.seg_blk.push_back(b);
                L.seg_j.push_back(L.bcol[b]);
                L.seg_slot.push_back(slot);
            }
            L.seg_ptr.push_back((int)L.seg_blk.size());
            for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b) {
                const bool live = L.bkind[b] == 0 || L.first_touch[b] < c;
                if (!live) continue;
                const int bt = L.btr[b];
                L.pj_box.push_back(i);
                L.pj_blk.push_back(b);
                L.pj_blkT.push_back(bt);
                auto& zb = L.bkind[b] == 1 ? L.zf_box : L.zn_box;
                auto& zk = L.bkind[b] == 1 ? L.zf_blk : L.zn_blk;
                auto& zc = L.bkind[b] == 1 ? L.zf_col : L.zn_col;
                zb.push_back(i); zk.push_back(b); zc.push_back(0);
                zb.push_back(i); zk.push_back(bt); zc.push_back(1);
            }
            ++slot;
        }
        L.seg_cptr.push_back((int)L.seg_blk.size());
        L.pj_cptr.push_back((int)L.pj_box.size());
        L.zf_cptr.push_back((int)L.zf_box.size());
        L.zn_cptr.push_back((int)L.zn_box.size());
    }
}

static int64_t adm_entry(const HostStructure& H, int64_t gs, int64_t gt) {
    auto b = H.adm_col.begin() + H.adm_ptr[gs];
    auto e = H.adm_col.begin() + H.adm_ptr[gs + 1];
    for (auto it = b; it != e; ++it)
        if (*it == gt) return (int64_t)(it - H.adm_col.begin());
    return -1;
}

// sources of each parent block from the four child pairs (level close)
static void close_lists(const HostStructure& H, LevelStruct& C, const LevelStruct& P) {
    int nb = P.nblocks();
    C.cl_dblk.assign(4 * (size_t)nb, -1);
    C.cl_fblk.assign(4 * (size_t)nb, -1);
    C.cl_adm.assign(4 * (size_t)nb, -1);
    parallel_for(P.cnt, [&](int64_t lo, int64_t hi) {
        for (int p = (int)lo; p < (int)hi; ++p)
            for (int b = P.bptr[p]; b < P.bptr[p + 1]; ++b) {
                int q = P.bcol[b];
                for (int a = 0; a < 2; ++a)
                    for (int bb = 0; bb < 2; ++bb) {
                        int c = 2 * p + a, e = 2 * q + bb;
                        int slot = 4 * b + 2 * a + bb;
                        int blk = C.find(c, e);
                        if (blk >= 0) {
                            if (C.bkind[blk] == 0) C.cl_dblk[slot] = blk;
                            else C.cl_fblk[slot] = blk;
                        }
                        C.cl_adm[slot] = adm_entry(H, C.first + c, C.first + e);
                    }
            }
    });
}

// leaf near blocks come from A's inadmissible leaf entries
static void leaf_entries(const HostStructure& H, LevelStruct& L) {
    L.near_entry.assign(L.nblocks(), -1);
    for (int i = 0; i < L.cnt; ++i) {
        if (L.state[i] == 0) continue;
        int64_t g = L.first + i;
        for (int64_t e = H.inad_ptr[g]; e < H.inad_ptr[g + 1]; ++e) {
            int j = (int)(H.inad_col[e] - L.first);
            L.near_entry[L.find(i, j)] = e - H.inad_ptr[L.first];
        }
    }
}

void build_plan(const HostStructure& H, Plan& P) {
    P.d = H.d;
    // per system: t_s = the coarsest level holding an admissible block (levels t_s ..
    // leaves are skeletonised; the dense top matrix is formed at level t_s - 1), or -1
    // when nothing is admissible (the top matrix is the leaf near field)
    P.sys_top.assign(H.nsys, -1);
    for (int64_t g = 0; g < H.nnodes; ++g)
        if (H.adm_ptr[g + 1] > H.adm_ptr[g]) {
            const int l = H.level_of(g);
            int& t = P.sys_top[H.sys[g]];
            t = t < 0 ? l : std::min(t, l);
        }
    P.sys_toplev.assign(H.nsys, H.d);
    P.top = -1;
    for (int s = 0; s < H.nsys; ++s)
        if (P.sys_top[s] >= 0) {
            P.sys_toplev[s] = P.sys_top[s] - 1;
            P.top = P.top < 0 ? P.sys_top[s] : std::min(P.top, P.sys_top[s]);
        }
    auto set_state = [&](LevelStruct& L, int l) {
        L.state.assign(H.lev_cnt[l], 0);
        for (int64_t i = 0; i < H.lev_cnt[l]; ++i) {
            const int s = H.sys[H.lev_first[l] + i];
            if (P.sys_top[s] >= 0 && l >= P.sys_top[s]) L.state[i] = 1;
            else if (l == P.sys_toplev[s]) L.state[i] = 2;
        }
    };
    P.levels.clear();
    std::vector<std::pair<int, int>> carried;
    int lowest = P.top < 0 ? H.d + 1 : P.top;       // forest levels with skeletonised boxes
    for (int l = H.d; l >= lowest; --l) {
        LevelStruct L;
        set_state(L, l);
        near_graph(H, l, L);
        colour_level(L);
        block_list(L, carried);
        schur_lists(L);
        solve_lists(L);
        work_lists(L);
        if (l == H.d) leaf_entries(H, L);
        else L.near_entry.assign(L.nblocks(), -1);
        // fill carried to the parent level: parents of fill pairs
        carried.clear();
        for (int i = 0; i < L.cnt; ++i)
            for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b)
                if (L.bkind[b] == 1) carried.push_back({i / 2, L.bcol[b] / 2});
        std::sort(carried.begin(), carried.end());
        carried.erase(std::unique(carried.begin(), carried.end()), carried.end());
        P.levels.push_back(std::move(L));
    }
    // the last level: dense top matrices only (t-1, or the leaves when no level is
    // skeletonised)
    int lt = P.top < 0 ? H.d : P.top - 1;
    LevelStruct T;
    set_state(T, lt);
    near_graph(H, lt, T);
    colour_level(T);
    block_list(T, P.top < 0 ? std::vector<std::pair<int, int>>{} : carried);
    if (P.top < 0) leaf_entries(H, T);
    else T.near_entry.assign(T.nblocks(), -1);
    P.toplev = std::move(T);
    // close lists: level l -> l-1 (parent of the last skeletonised level is toplev)
    for (size_t a = 0; a < P.levels.size(); ++a) {
        const LevelStruct& par = (a + 1 < P.levels.size()) ? P.levels[a + 1] : P.toplev;
        close_lists(H, P.levels[a], par);
    }
}

static void upload_level(LevelStruct& L, cudaStream_t s) {
    std::vector<int> brow(L.nblocks()), diag(L.cnt, -1);
    for (int i = 0; i < L.cnt; ++i) {
        for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b) brow[b] = i;
        diag[i] = L.find(i, i);
    }
    std::vector<int> all;
    L.cbox_ptr.assign(1, 0);
    for (auto& cb : L.cboxes) {
        all.insert(all.end(), cb.begin(), cb.end());
        L.cbox_ptr.push_back((int)all.size());
    }
    LevelStruct::Dev& d = L.dev;
    upload(d.colour, L.colour, s);
    upload(d.brow, brow, s);
    upload(d.bcol, L.bcol, s);
    upload(d.top_boxes, L.top_boxes, s);
    upload(d.skel_boxes, L.skel_boxes, s);
    upload(d.nb_ptr, L.nb_ptr, s);
    upload(d.nb_col, L.nb_col, s);
    upload(d.nb_blk, L.nb_blk, s);
    upload(d.nb_blkT, L.nb_blkT, s);
    upload(d.diag_blk, diag, s);
    upload(d.fl_tbox, L.fl_tbox, s);
    upload(d.fl_tptr, L.fl_tptr, s);
    upload(d.fl_ci, L.fl_ci, s);
    upload(d.fl_cpos, L.fl_cpos, s);
    upload(d.near_entry, L.near_entry, s);
    upload(d.sch_tblk, L.sch_tblk, s);
    upload(d.sch_tptr, L.sch_tptr, s);
    upload(d.sch_ci, L.sch_ci, s);
    upload(d.sch_cA, L.sch_cA, s);
    upload(d.sch_ckpos, L.sch_ckpos, s);
    upload(d.cl_dblk, L.cl_dblk, s);
    upload(d.cl_fblk, L.cl_fblk, s);
    upload(d.cl_adm, L.cl_adm, s);
    upload(d.cboxes, all, s);
    upload(d.seg_blk, L.seg_blk, s);
    upload(d.seg_j, L.seg_j, s);
    upload(d.seg_slot, L.seg_slot, s);
    upload(d.seg_ptr, L.seg_ptr, s);
    upload(d.pj_box, L.pj_box, s);
    upload(d.pj_blk, L.pj_blk, s);
    upload(d.pj_blkT, L.pj_blkT, s);
    upload(d.zf_box, L.zf_box, s);
    upload(d.zf_blk, L.zf_blk, s);
    upload(d.zf_col, L.zf_col, s);
    upload(d.zn_box, L.zn_box, s);
    upload(d.zn_blk, L.zn_blk, s);
    upload(d.zn_col, L.zn_col, s);
}

void upload_plan(Plan& P, cudaStream_t s) {
    for (auto& L : P.levels) upload_level(L, s);
    upload_level(P.toplev, s);
}

}  // namespace h2rs
