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
#include <atomic>
#include <exception>
#include <mutex>
#include <thread>

#include "h2rs_internal.h"

namespace h2rs {

// job(t) for t in [0, nt): t = 0 on the calling thread, the others on their own
// threads (inline when no thread can be had).  An exception thrown by any job (a
// failed host allocation, an invalid structure) is rethrown here once all have joined.
template <class J>
static void run_threads(int64_t nt, J job) {
    std::exception_ptr err;
    std::mutex mu;
    auto guarded = [&](int64_t t) {
        try {
            job(t);
        } catch (...) {
            std::lock_guard<std::mutex> g(mu);
            if (!err) err = std::current_exception();
        }
    };
    std::vector<std::thread> th;
    for (int64_t t = 1; t < nt; ++t) {
        try {
            th.emplace_back(guarded, t);
        } catch (...) {
            guarded(t);
        }
    }
    guarded(0);
    for (auto& x : th) x.join();
    if (err) std::rethrow_exception(err);
}

static int64_t host_threads() {
    return std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), 32);
}

// f(lo, hi) over [0, n) in contiguous ranges on the host's cores (the plan of a
// million-point matrix walks tens of millions of block pairs), at least `grain` items
// per thread
template <class F>
static void parallel_for(int64_t n, F f, int64_t grain = 16) {
    const int64_t nt = std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / grain));
    if (nt <= 1) {
        f((int64_t)0, n);
        return;
    }
    run_threads(nt, [&](int64_t t) { f(n * t / nt, n * (t + 1) / nt); });
}

// f(item, scratch) for every item in [0, n), handed out one at a time to the host's
// cores (for items of very different cost, e.g. colours); each thread owns one S
template <class S, class F>
static void parallel_items(int64_t n, F f) {
    const int64_t nt = std::min<int64_t>(host_threads(), n);
    std::atomic<int64_t> next{0};
    run_threads(nt, [&](int64_t) {
        S scratch;
        for (int64_t c; (c = next.fetch_add(1)) < n;) f(c, scratch);
    });
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

static void atomic_min(int* p, int v) {
    int cur = __atomic_load_n(p, __ATOMIC_RELAXED);
    while (v < cur && !__atomic_compare_exchange_n(p, &cur, v, true, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
    }
}

// Schur targets per colour (target-owned accumulation) and first touches of fill;
// the colours are listed concurrently, then concatenated in colour order.  Within a
// colour the targets are ascending and each target's contributors ascending in i: the
// contributions are generated box by box (boxes ascending) and bucketed by target.
static void schur_lists(LevelStruct& L) {
    struct Part {
        std::vector<int> tblk, tlen, ci, cA, ckpos, cjpos;
    };
    struct Scratch {
        std::vector<int> cnt, pos, rt, ri, ra, rk, rj;
    };
    std::vector<Part> parts(L.ncolour);
    const int nb = L.nblocks();
    parallel_items<Scratch>(L.ncolour, [&](int64_t c, Scratch& s) {
        if ((int)s.cnt.size() != nb) {
            s.cnt.assign(nb, 0);
            s.pos.resize(nb);
        }
        s.rt.clear(); s.ri.clear(); s.ra.clear(); s.rk.clear(); s.rj.clear();
        for (int i : L.cboxes[c]) {
            const int n0 = L.nb_ptr[i], n1 = L.nb_ptr[i + 1];
            for (int a = n0; a < n1; ++a) {
                const int j = L.nb_col[a];
                const int ablk = L.find(j, i);
                // every k in N(i) is a block of row j (near field or fill): walk the row
                int p = L.bptr[j];
                const int pe = L.bptr[j + 1];
                for (int b = n0; b < n1; ++b) {
                    const int k = L.nb_col[b];
                    while (p < pe && L.bcol[p] < k) ++p;
                    H2_REQUIRE(p < pe && L.bcol[p] == k && ablk >= 0, H2_ERR_ARG,
                               "the near field is not symmetric");
                    ++s.cnt[p];
                    s.rt.push_back(p);
                    s.ri.push_back(i);
                    s.ra.push_back(ablk);
                    s.rk.push_back(b - n0);
                    s.rj.push_back(a - n0);
                }
            }
        }
        Part& P = parts[c];
        int run = 0;
        for (int t = 0; t < nb; ++t)
            if (s.cnt[t]) {
                P.tblk.push_back(t);
                P.tlen.push_back(s.cnt[t]);
                s.pos[t] = run;
                run += s.cnt[t];
                s.cnt[t] = 0;
            }
        P.ci.resize(run);
        P.cA.resize(run);
        P.ckpos.resize(run);
        P.cjpos.resize(run);
        for (size_t r = 0; r < s.rt.size(); ++r) {
            const int q = s.pos[s.rt[r]]++;
            P.ci[q] = s.ri[r];
            P.cA[q] = s.ra[r];
            P.ckpos[q] = s.rk[r];
            P.cjpos[q] = s.rj[r];
        }
    });
    // concatenation in colour order: sizes first, then every colour copied in parallel
    const int nc = L.ncolour;
    L.sch_cptr.assign(nc + 1, 0);
    std::vector<int> coff(nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        L.sch_cptr[c + 1] = L.sch_cptr[c] + (int)parts[c].tblk.size();
        coff[c + 1] = coff[c] + (int)parts[c].ci.size();
    }
    L.sch_tblk.resize(L.sch_cptr[nc]);
    L.sch_tptr.resize(L.sch_cptr[nc] + 1);
    L.sch_tptr[0] = 0;
    L.sch_ci.resize(coff[nc]);
    L.sch_cA.resize(coff[nc]);
    L.sch_ckpos.resize(coff[nc]);
    L.sch_cjpos.resize(coff[nc]);
    parallel_items<int>(nc, [&](int64_t c, int&) {
        const Part& P = parts[c];
        const int t0 = L.sch_cptr[c];
        int run = coff[c];
        for (size_t q = 0; q < P.tblk.size(); ++q) {
            L.sch_tblk[t0 + q] = P.tblk[q];
            run += P.tlen[q];
            L.sch_tptr[t0 + q + 1] = run;
        }
        std::copy(P.ci.begin(), P.ci.end(), L.sch_ci.begin() + coff[c]);
        std::copy(P.cA.begin(), P.cA.end(), L.sch_cA.begin() + coff[c]);
        std::copy(P.ckpos.begin(), P.ckpos.end(), L.sch_ckpos.begin() + coff[c]);
        std::copy(P.cjpos.begin(), P.cjpos.end(), L.sch_cjpos.begin() + coff[c]);
    });
    // a fill block is first touched by the first (lowest) colour that updates it;
    // blocks carried from the level below keep -1
    parallel_items<int>(nc, [&](int64_t c, int&) {
        for (int t : parts[c].tblk)
            if (L.bkind[t] == 1) atomic_min(&L.first_touch[t], (int)c);
    });
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
    // per colour: targets j ascending, each with its contributors i ascending
    struct Part {
        std::vector<int> tbox, tlen, ci, cpos;
    };
    std::vector<Part> parts(L.ncolour);
    struct Rec { int j, i, pos; };
    parallel_items<std::vector<Rec>>(L.ncolour, [&](int64_t c, std::vector<Rec>& recs) {
        recs.clear();
        for (int i : L.cboxes[c])
            for (int a = L.nb_ptr[i]; a < L.nb_ptr[i + 1]; ++a)
                recs.push_back({L.nb_col[a], i, a - L.nb_ptr[i]});
        std::sort(recs.begin(), recs.end(), [](const Rec& x, const Rec& y) {
            return x.j != y.j ? x.j < y.j : x.i < y.i;
        });
        Part& P = parts[c];
        for (size_t r = 0; r < recs.size(); ++r) {
            if (r == 0 || recs[r].j != recs[r - 1].j) {
                P.tbox.push_back(recs[r].j);
                P.tlen.push_back(0);
            }
            ++P.tlen.back();
            P.ci.push_back(recs[r].i);
            P.cpos.push_back(recs[r].pos);
        }
    });
    L.fl_cptr.assign(1, 0);
    L.fl_tbox.clear();
    L.fl_tptr.assign(1, 0);
    L.fl_ci.clear();
    L.fl_cpos.clear();
    for (const Part& P : parts) {
        for (size_t q = 0; q < P.tbox.size(); ++q) {
            L.fl_tbox.push_back(P.tbox[q]);
            L.fl_tptr.push_back(L.fl_tptr.back() + P.tlen[q]);
        }
        L.fl_ci.insert(L.fl_ci.end(), P.ci.begin(), P.ci.end());
        L.fl_cpos.insert(L.fl_cpos.end(), P.cpos.begin(), P.cpos.end());
        L.fl_cptr.push_back((int)L.fl_tbox.size());
    }
}

// structure-only work lists of every colour (first_touch is final after schur_lists);
// built per colour in parallel, then concatenated in colour order
static void work_lists(LevelStruct& L) {
    struct Part {
        std::vector<int> seg_blk, seg_j, seg_slot, seg_end;      // seg_end: local end per box
        std::vector<int> pj_box, pj_blk, pj_blkT;
        std::vector<int> zf_box, zf_blk, zf_col, zn_box, zn_blk, zn_col;
        std::vector<int> pk_box, pk_pos;
        std::vector<int> pj_end;                                 // local end of each box's entries
    };
    std::vector<Part> parts(L.ncolour);
    parallel_items<int>(L.ncolour, [&](int64_t c64, int&) {
        const int c = (int)c64;
        Part& P = parts[c];
        int slot = 0;
        for (int i : L.cboxes[c]) {
            for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b) {
                if (L.bkind[b] != 1 || L.first_touch[b] >= c) continue;
                P.seg_blk.push_back(b);
                P.seg_j.push_back(L.bcol[b]);
                P.seg_slot.push_back(slot);
            }
            P.seg_end.push_back((int)P.seg_blk.size());
            for (int a = L.nb_ptr[i]; a < L.nb_ptr[i + 1]; ++a) {
                P.pk_box.push_back(i);
                P.pk_pos.push_back(a);
            }
            for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b) {
                const bool live = L.bkind[b] == 0 || L.first_touch[b] < c;
                if (!live) continue;
                const int bt = L.btr[b];
                P.pj_box.push_back(i);
                P.pj_blk.push_back(b);
                P.pj_blkT.push_back(bt);
                auto& zb = L.bkind[b] == 1 ? P.zf_box : P.zn_box;
                auto& zk = L.bkind[b] == 1 ? P.zf_blk : P.zn_blk;
                auto& zc = L.bkind[b] == 1 ? P.zf_col : P.zn_col;
                zb.push_back(i); zk.push_back(b); zc.push_back(0);
                zb.push_back(i); zk.push_back(bt); zc.push_back(1);
            }
            P.pj_end.push_back((int)P.pj_box.size());
            ++slot;
        }
    });
    L.seg_blk.clear(); L.seg_j.clear(); L.seg_slot.clear();
    L.seg_ptr.assign(1, 0);
    L.seg_cptr.assign(1, 0);
    L.pj_box.clear(); L.pj_blk.clear(); L.pj_blkT.clear();
    L.pj_cptr.assign(1, 0);
    L.zf_box.clear(); L.zf_blk.clear(); L.zf_col.clear();
    L.zn_box.clear(); L.zn_blk.clear(); L.zn_col.clear();
    L.zf_cptr.assign(1, 0);
    L.zn_cptr.assign(1, 0);
    L.pk_box.clear(); L.pk_pos.clear();
    L.pk_cptr.assign(1, 0);
    L.pj_ptr.assign(1, 0);
    auto append = [](std::vector<int>& dst, const std::vector<int>& src) { dst.insert(dst.end(), src.begin(), src.end()); };
    for (const Part& P : parts) {
        const int base = (int)L.seg_blk.size();
        for (int e : P.seg_end) L.seg_ptr.push_back(base + e);
        const int pbase = (int)L.pj_box.size();
        for (int e : P.pj_end) L.pj_ptr.push_back(pbase + e);
        append(L.seg_blk, P.seg_blk); append(L.seg_j, P.seg_j); append(L.seg_slot, P.seg_slot);
        append(L.pj_box, P.pj_box); append(L.pj_blk, P.pj_blk); append(L.pj_blkT, P.pj_blkT);
        append(L.zf_box, P.zf_box); append(L.zf_blk, P.zf_blk); append(L.zf_col, P.zf_col);
        append(L.zn_box, P.zn_box); append(L.zn_blk, P.zn_blk); append(L.zn_col, P.zn_col);
        append(L.pk_box, P.pk_box); append(L.pk_pos, P.pk_pos);
        L.pk_cptr.push_back((int)L.pk_box.size());
        L.seg_cptr.push_back((int)L.seg_blk.size());
        L.pj_cptr.push_back((int)L.pj_box.size());
        L.zf_cptr.push_back((int)L.zf_box.size());
        L.zn_cptr.push_back((int)L.zn_box.size());
    }
}

// sources of each parent block from the four child pairs (level close).  A child
// pair (c, e) that is admissible takes its coupling from A's admissible CSR: the first
// entry of row c with column e (each child row's entries are sorted by column once)
static void close_lists(const HostStructure& H, LevelStruct& C, const LevelStruct& P) {
    int nb = P.nblocks();
    C.cl_dblk.assign(4 * (size_t)nb, -1);
    C.cl_fblk.assign(4 * (size_t)nb, -1);
    C.cl_adm.assign(4 * (size_t)nb, -1);
    parallel_for(P.cnt, [&](int64_t lo, int64_t hi) {
        std::vector<std::pair<int64_t, int64_t>> row[2];      // (column, entry) of rows 2p, 2p+1
        for (int p = (int)lo; p < (int)hi; ++p) {
            for (int a = 0; a < 2; ++a) {
                const int64_t g = C.first + 2 * p + a;
                row[a].clear();
                for (int64_t e = H.adm_ptr[g]; e < H.adm_ptr[g + 1]; ++e) row[a].push_back({H.adm_col[e], e});
                std::sort(row[a].begin(), row[a].end());
            }
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
                        const int64_t ge = C.first + e;
                        auto it = std::lower_bound(row[a].begin(), row[a].end(), std::make_pair(ge, (int64_t)INT64_MIN));
                        if (it != row[a].end() && it->first == ge) C.cl_adm[slot] = it->second;
                    }
            }
        }
    });
}

// leaf near blocks come from A's inadmissible leaf entries
static void leaf_entries(const HostStructure& H, LevelStruct& L) {
    L.near_entry.assign(L.nblocks(), -1);
    parallel_for(L.cnt, [&](int64_t lo, int64_t hi) {
        for (int i = (int)lo; i < (int)hi; ++i) {
            if (L.state[i] == 0) continue;
            int64_t g = L.first + i;
            for (int64_t e = H.inad_ptr[g]; e < H.inad_ptr[g + 1]; ++e) {
                int j = (int)(H.inad_col[e] - L.first);
                L.near_entry[L.find(i, j)] = e - H.inad_ptr[L.first];
            }
        }
    });
}

// fill carried to the parent level: the parent pairs (i/2, j/2) of the fill blocks,
// sorted and distinct (gathered per parent row: its two child rows)
static void carried_pairs(const LevelStruct& L, std::vector<std::pair<int, int>>& out) {
    const int np = (L.cnt + 1) / 2;
    std::vector<std::vector<int>> rows(np);
    parallel_for(np, [&](int64_t lo, int64_t hi) {
        for (int p = (int)lo; p < (int)hi; ++p) {
            auto& r = rows[p];
            for (int i = 2 * p; i < std::min(2 * p + 2, L.cnt); ++i)
                for (int b = L.bptr[i]; b < L.bptr[i + 1]; ++b)
                    if (L.bkind[b] == 1) r.push_back(L.bcol[b] / 2);
            std::sort(r.begin(), r.end());
            r.erase(std::unique(r.begin(), r.end()), r.end());
        }
    });
    out.clear();
    for (int p = 0; p < np; ++p)
        for (int q : rows[p]) out.push_back({p, q});
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
        carried_pairs(L, carried);
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
    upload(d.sch_cjpos, L.sch_cjpos, s);
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
    upload(d.pj_ptr, L.pj_ptr, s);
    upload(d.zf_box, L.zf_box, s);
    upload(d.zf_blk, L.zf_blk, s);
    upload(d.zf_col, L.zf_col, s);
    upload(d.zn_box, L.zn_box, s);
    upload(d.zn_blk, L.zn_blk, s);
    upload(d.zn_col, L.zn_col, s);
    upload(d.pk_box, L.pk_box, s);
    upload(d.pk_pos, L.pk_pos, s);
}

void upload_plan(Plan& P, cudaStream_t s) {
    for (auto& L : P.levels) upload_level(L, s);
    upload_level(P.toplev, s);
}

}  // namespace h2rs
