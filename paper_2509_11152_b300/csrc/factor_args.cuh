// Device kernels of the factorisation (templated on the working type T).
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "h2rs_internal.h"

namespace h2rs {

template <class T> struct Eps;
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };
template <> struct Eps<float> { static constexpr float v = FLT_EPSILON; };

// Per-level device view shared by the kernels.
template <class T>
struct LevelArgs {
    int level;
    int cnt;
    const int* n;          // box sizes
    const int* k;          // basis ranks before augmentation
    int* kt;               // augmented ranks (written by the basis kernel)
    const int* colour;
    const int64_t* blk_off;
    const int* brow;
    const int* bcol;
    T* blk;
    const int64_t* V_off;
    const T* V;
    const int64_t* Q_off;
    T* Q;
    const int64_t* LU_off;
    T* LU;
    T* DI;                 // D_RR^-1 per box (same offsets as Q)
    const int64_t* piv_off;
    int* piv;
    const int64_t* WU_off;
    T* WU;
    const int64_t* WL_off;
    T* WL;
    const int* WLld;
    const int* nb_ptr;
    const int* nb_col;
    const int* nbofs;      // column offset of neighbour (by N(i) position) in W_U^i
    const int* Nsum;       // sum of n_j over N(i) without i
    const int* nb_blk;     // block id of (i, j) per N(i) position
    const int* nb_blkT;    // block id of (j, i) per N(i) position
    const int* diag_blk;   // block id of (i, i)
    const T* eps_fill;     // truncation threshold eps_lu * ||A_s|| of every box
    const int* force_kt;   // debug: forced augmented ranks of the level, or null
    DevStatus* status;
};

// One dense top matrix of the batch (float64, column-major nt x nt) and its pivots.
struct TopSys {
    double* A;
    int* piv;
    int64_t nt;
};

// Schur update records, filled per colour once the colour's ranks and W_U are known
// (so that a tile walks one record per contributor instead of a chain of index loads).
struct SchurCon {
    int64_t aoff;          // byte offset of the packed D_{j,i_R} region (A operand)
    int64_t boff;          // byte offset of the packed W_U^i[k] region (B operand)
    int ri;                // redundant size of contributor i (0: nothing to add)
    int pad;
};
struct SchurTgt {
    int64_t coff;          // element offset of the target's first updated entry in blk
    int nj;                // leading dimension (rows of the target block)
    int m, nn;             // updated rows / columns
    int row_lo;            // first updated row
    int cb, ce;            // contributor records cb .. ce-1
    int nsl;               // K slices of 16 over all contributors
    int ga, gb;            // row groups per part of a packed slice: ceil(n_j / 8), ceil(n_k / 8)
    SchurCon c0;           // copy of record cb (read with the target: one load less)
};

// Per-colour work lists of the basis kernels (device pointers).
struct ColourLists {
    const int* boxes;          // boxes of the colour
    const int* seg_ptr;        // nbox+1: fill segments of each box
    const int* seg_blk;        // fill block (i, j)
    const int* seg_j;          // column box j
    const int64_t* ybase;      // scratch offset of the box's Y^T
    const int64_t* ylead;      // leading dimension (total rows) of the box's Y^T
    const int64_t* wbase;      // scratch offset of the box's n x n work matrix
    double* ynorm2;            // ||Y||_F^2 of the box's fill rows (zero before the gather)
};

}  // namespace h2rs
