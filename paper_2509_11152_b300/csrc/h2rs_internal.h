// Internal declarations of the h2rs library (not part of the public C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/h2rs.h"

namespace h2rs {

// ------------------------------------------------------------------ errors
struct Error {
    int code;
    std::string msg;
};

void set_error(const std::string& msg);

// process-wide count of kernel launches (h2_kernel_launch_count)
void count_launch(int64_t n = 1);

#define H2_CUDA_CHECK(call)                                                          \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            throw ::h2rs::Error{H2_ERR_CUDA, std::string(#call) + ": " +             \
                                                 cudaGetErrorString(e_)};            \
    } while (0)

#define H2_REQUIRE(cond, code, msg)                                                  \
    do {                                                                             \
        if (!(cond)) throw ::h2rs::Error{(code), (msg)};                            \
    } while (0)

// Runs f and turns every exception into a status code (and h2_last_error's message):
// nothing is thrown across the C-ABI.
template <class F>
int guard(F&& f) {
    try {
        f();
        return H2_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return H2_ERR_OOM;
    } catch (const std::exception& e) {
        set_error(e.what());
        return H2_ERR_ARG;
    } catch (...) {
        set_error("unknown error");
        return H2_ERR_ARG;
    }
}

// device status word written by kernels (never trapped on)
struct DevStatus {
    int code;       // 0 ok, else an H2_ERR_* value
    int level;
    int box;
    int pad;
};

// ------------------------------------------------------------------ memory
// Stream-ordered device buffer (cudaMallocAsync from the default pool).
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
    DevBuf& operator=(DevBuf&& o) noexcept {
        release();
        ptr = o.ptr; bytes = o.bytes; stream = o.stream;
        o.ptr = nullptr; o.bytes = 0;
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t nbytes, cudaStream_t s);
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// non-owning view of device memory owned elsewhere (same accessor as DevBuf)
struct DevView {
    void* ptr = nullptr;
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// upload a host vector into a fresh device buffer
template <class T>
void upload(DevBuf& b, const std::vector<T>& v, cudaStream_t s) {
    b.alloc(std::max<size_t>(1, v.size()) * sizeof(T), s);
    if (!v.empty())
        H2_CUDA_CHECK(cudaMemcpyAsync(b.ptr, v.data(), v.size() * sizeof(T),
                                      cudaMemcpyHostToDevice, s));
}

// ------------------------------------------------------------------ host copy of A
// A forest of one or more complete binary cluster trees whose levels are aligned by
// height above the leaves (a batch of independent systems).  Level l (0 = the roots
// of the deepest trees, d = every leaf) holds the global node ids
// lev_first[l] .. lev_first[l] + lev_cnt[l] - 1; trees are ordered by decreasing depth
// so that the children of local box i at level l are the local boxes 2i and 2i+1 at
// level l+1, and a tree of depth d_s has its root at level d - d_s.  For one tree this
// is the heap numbering (lev_first[l] = 2^l - 1).
struct HostStructure {
    int64_t n = 0;
    int d = 0;
    int64_t nnodes = 0;
    std::vector<int64_t> node_start, node_size, rank;
    std::vector<int64_t> U_off, E_off, adm_ptr, adm_col, S_off, inad_ptr, inad_col, D_off;
    std::vector<int64_t> lev_first, lev_cnt;  // d+1 entries
    std::vector<int64_t> parent;              // global parent id, -1 for a root
    std::vector<int> sys;                     // system (tree) of every node
    int nsys = 1;
    std::vector<int> sys_root;                // level of each system's root
    std::vector<int64_t> sys_voff;            // nsys+1: vector offsets (caller order)
    int level_of(int64_t g) const;            // level of a global node id
};

// ------------------------------------------------------------------ plan
// Structure-only (rank independent) plan of one level, built once per matrix.
struct LevelStruct {
    int l = 0;
    int cnt = 0;               // boxes at the level
    int64_t first = 0;         // global id of the first box
    // box state: 0 not reached (above its system's top), 1 skeletonised at this level,
    // 2 part of its system's dense top matrix
    std::vector<int8_t> state;
    std::vector<int> top_boxes;               // boxes with state 2, ascending
    std::vector<int> skel_boxes;              // boxes with state 1, ascending
    std::vector<int> nb_ptr, nb_col;          // near field N(i), sorted, includes i
    std::vector<int> colour;
    int ncolour = 0;
    std::vector<std::vector<int>> cboxes;     // boxes of each colour, ascending
    // merged block list: near field + fill pattern, CSR, columns ascending
    std::vector<int> bptr, bcol;
    std::vector<int8_t> bkind;                // 0 near, 1 fill
    std::vector<int> btr;                     // index of the transposed block
    std::vector<int> first_touch;             // fill: -1 carried, c = first colour
                                              // writing it, INT_MAX never
    std::vector<int64_t> near_entry;          // near block -> entry of A's inad CSR
    // Schur target lists, per colour: targets (block ids) and their contributors
    std::vector<int> sch_cptr;                // ncolour+1 -> ranges of targets
    std::vector<int> sch_tblk;                // target block
    std::vector<int> sch_tptr;                // ntargets+1 -> ranges of contributors
    std::vector<int> sch_ci;                  // contributor box i
    std::vector<int> sch_cA;                  // block (j, i)  (A operand)
    std::vector<int> sch_ckpos;               // position of k in N(i)
    std::vector<int> sch_cjpos;               // position of j in N(i)
    // per near-field position (nb_ptr order): block ids of (i, j) and (j, i)
    std::vector<int> nb_blk, nb_blkT;
    // per-colour work lists (boxes in cboxes order): fill segments of the basis
    // augmentation (seg_slot = box position in its colour, seg_ptr = per box, global),
    // live blocks to project (row block b and its transpose), blocks to zero
    std::vector<int> seg_blk, seg_j, seg_slot, seg_ptr, seg_cptr;
    std::vector<int> pj_box, pj_blk, pj_blkT, pj_cptr;
    std::vector<int> pj_ptr;                  // per box (cboxes order): its first pj entry (+ end)
    std::vector<int> zf_box, zf_blk, zf_col, zf_cptr, zn_box, zn_blk, zn_col, zn_cptr;
    // operand packing of the tensor-core Schur update: every near-field position p of
    // every box i of the colour (box, position), per colour
    std::vector<int> pk_box, pk_pos, pk_cptr;
    // forward-solve L updates, per colour: target boxes j and contributors i
    std::vector<int> fl_cptr;                 // ncolour+1 -> ranges of targets
    std::vector<int> fl_tbox;                 // target box j
    std::vector<int> fl_tptr;                 // ntargets+1 -> ranges of contributors
    std::vector<int> fl_ci;                   // contributor box i
    std::vector<int> fl_cpos;                 // position of j in N(i)
    // level close to the parent level (l-1): per parent block, 4 child sources
    std::vector<int> cl_dblk;                 // 4 per parent block, near block or -1
    std::vector<int> cl_fblk;                 // 4 per parent block, fill block or -1
    std::vector<int64_t> cl_adm;              // 4 per parent block, adm entry or -1

    int find(int i, int j) const;             // merged block id of (i, j) or -1
    int nblocks() const { return (int)bcol.size(); }

    // device copies of the structure above, uploaded once with the matrix
    struct Dev {
        DevBuf colour, brow, bcol, top_boxes, skel_boxes, nb_ptr, nb_col, nb_blk, nb_blkT, diag_blk;
        DevBuf fl_tbox, fl_tptr, fl_ci, fl_cpos, near_entry;
        DevBuf sch_tblk, sch_tptr, sch_ci, sch_cA, sch_ckpos, sch_cjpos, cl_dblk, cl_fblk, cl_adm;
        DevBuf cboxes;                        // boxes of every colour, in colour order
        DevBuf seg_blk, seg_j, seg_slot, seg_ptr, pj_box, pj_blk, pj_blkT, pj_ptr;
        DevBuf zf_box, zf_blk, zf_col, zn_box, zn_blk, zn_col, pk_box, pk_pos;
    } dev;
    std::vector<int> cbox_ptr;                // ncolour+1 offsets into dev.cboxes
};

struct Plan {
    int d = 0;
    int top = -1;                             // min over systems of t, -1 when no system
                                              // has an admissible block
    std::vector<int> sys_top;                 // per system: t_s (forest level), or -1
    std::vector<int> sys_toplev;              // per system: level of its dense top matrix
    std::vector<LevelStruct> levels;          // index 0 = level d (leaves) ... level top
    LevelStruct toplev;                       // the last level: dense top matrices only
};

void build_plan(const HostStructure& H, Plan& P);
// device copies of every level's structure (LevelStruct::dev)
void upload_plan(Plan& P, cudaStream_t s);

// one tree (heap numbering) from a descriptor, with consistency checks
void read_structure(const h2_matrix_desc* d, HostStructure& H);
// Where each tree's value arrays (U, E, S, D) land in the forest's arrays: element
// ranges copied unchanged (a tree's values of one level stay contiguous).
struct ValueChunk {
    int sys;                                  // caller index of the tree
    int64_t src, dst, cnt;                    // element offsets and count
};
struct ForestValues {
    std::vector<ValueChunk> U, E, S, D;
};
// forest of the trees in `parts` (caller order); order[r] = caller index of the tree at
// merged rank r (trees sorted by decreasing depth, ties in caller order)
void merge_forest(const std::vector<HostStructure>& parts, HostStructure& F, std::vector<int>& order,
                  ForestValues& values);

// ------------------------------------------------------------------ objects
struct MatrixObj {
    HostStructure H;
    Plan plan;
    int device = 0;                           // device current at creation (holds the copies)
    cudaStream_t stream = nullptr;
    DevBuf U, E, S, D;                        // float64 values on the device
    DevBuf d_node_start, d_node_size, d_rank, d_U_off, d_E_off, d_S_off, d_D_off;
    DevBuf d_adm_ptr, d_adm_col, d_inad_ptr, d_inad_col;
    DevBuf d_parent;                          // forest parent of every node (-1: root)
    DevBuf d_child0;                          // first child id (children c, c+1), -1: leaf
    DevBuf d_sys_voff;                        // nsys+1 vector offsets of the systems
    // matvec helpers: per node offsets of the coefficient vectors (rank prefix)
    std::vector<int64_t> coef_off;
    DevBuf d_coef_off;
};

}  // namespace h2rs

struct h2_matrix {
    h2rs::MatrixObj m;
};
