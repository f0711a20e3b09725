/* Plain-C use of the h2rs C-ABI: a hand-built H^2 matrix descriptor and the host-only
 * plan query (no GPU needed).  The matrix: n = 8 points, depth 2 (root, 2 boxes,
 * 4 leaves of 2 points), rank-1 bases everywhere; at level 2 the leaf pairs (0,2),
 * (0,3), (1,3) and their transposes are admissible, every other pair is near field.
 * Values are placeholders (only the index arrays are read by the plan query).
 *
 * Build: cc plan_query.c -I<repo>/include -L<dir of libh2rs.so> -lh2rs -o plan_query
 */
#include <stdio.h>
#include <stdlib.h>

#include "h2rs.h"

int main(void) {
    enum { NN = 7, NLEAF = 4 };
    /* heap numbering: 0 root; 1, 2 level 1; 3..6 leaves */
    int64_t node_start[NN] = {0, 0, 4, 0, 2, 4, 6};
    int64_t node_size[NN] = {8, 4, 4, 2, 2, 2, 2};
    int64_t rank[NN] = {1, 1, 1, 1, 1, 1, 1};
    int64_t U_off[NLEAF + 1] = {0, 2, 4, 6, 8};             /* 2 x 1 per leaf */
    int64_t E_off[NN + 1] = {0, 0, 1, 2, 3, 4, 5, 6};        /* 1 x 1 per non-root */
    /* admissible pairs: level 2 only, leaves 3..6: (3,5) (3,6) (4,6) + transposes */
    int64_t adm_ptr[NN + 1] = {0, 0, 0, 0, 2, 3, 4, 6};
    int64_t adm_col[6] = {5, 6, 6, 3, 3, 4};
    int64_t S_off[7] = {0, 1, 2, 3, 4, 5, 6};
    /* inadmissible: root (0,0); level 1 all pairs; leaves: self + (3,4) (4,5) (5,6) */
    int64_t inad_ptr[NN + 1] = {0, 1, 3, 5, 7, 10, 13, 15};
    int64_t inad_col[15] = {0, 1, 2, 1, 2, 3, 4, 3, 4, 5, 4, 5, 6, 5, 6};
    int64_t D_off[11] = {0, 4, 8, 12, 16, 20, 24, 28, 32, 36, 40};   /* 10 leaf entries, 2 x 2 */
    double vals[64] = {0};
    h2_matrix_desc d = {0};
    d.n = 8;
    d.depth = 2;
    d.values_on_device = 0;
    d.node_start = node_start;
    d.node_size = node_size;
    d.rank = rank;
    d.U_off = U_off;
    d.U = vals;
    d.E_off = E_off;
    d.E = vals;
    d.adm_ptr = adm_ptr;
    d.adm_col = adm_col;
    d.S_off = S_off;
    d.S = vals;
    d.inad_ptr = inad_ptr;
    d.inad_col = inad_col;
    d.D_off = D_off;
    d.D = vals;

    printf("%s\n", h2_version());
    int64_t nbox = 0, nblk = 0;
    int rc = h2_plan_query(&d, 0, &nbox, &nblk, NULL, NULL, NULL, NULL);
    if (rc != H2_OK) {
        fprintf(stderr, "plan query failed (%d): %s\n", rc, h2_last_error());
        return 1;
    }
    int32_t colour[4];
    int64_t row_ptr[5];
    int64_t* col = (int64_t*)malloc(sizeof(int64_t) * (size_t)nblk);
    int32_t* kind = (int32_t*)malloc(sizeof(int32_t) * (size_t)nblk);
    rc = h2_plan_query(&d, 0, NULL, NULL, colour, row_ptr, col, kind);
    if (rc != H2_OK) return 1;
    printf("leaf level: %lld boxes, %lld blocks\n", (long long)nbox, (long long)nblk);
    for (int i = 0; i < (int)nbox; ++i) {
        printf("box %d colour %d:", i, colour[i]);
        for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b)
            printf(" %lld%s", (long long)col[b], kind[b] ? "f" : "");
        printf("\n");
    }
    /* a descriptor error is a status code, never a crash */
    node_size[1] = 5;
    rc = h2_plan_query(&d, 0, &nbox, &nblk, NULL, NULL, NULL, NULL);
    printf("bad descriptor: %d (%s)\n", rc, h2_last_error());
    free(col);
    free(kind);
    return rc == H2_ERR_ARG ? 0 : 1;
}
