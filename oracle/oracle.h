/* Oracle (test infrastructure only): declarations of the CPU definitions in
 * oracle.c.  Not included by, and shares nothing with, the GPU library. */
#pragma once
#include <stdint.h>

#define OR_MAX_DIMS 8
#define OR_MAX_PREDS 8

enum { OR_BETWEEN = 0, OR_EQ = 1, OR_NE = 2, OR_LT = 3, OR_LE = 4, OR_GT = 5, OR_GE = 6 };
enum { OR_AGG_COUNT = 0, OR_AGG_SUM = 1, OR_AGG_MUL = 2, OR_AGG_SUB = 3 };
enum { OR_E_DUPKEY = -10, OR_E_RANGE = -11, OR_E_NOMEM = -12 };

typedef struct {
  const int32_t *col; /* fact column (n rows) */
  int32_t op, lo, hi;
} or_pred;

typedef struct {
  const int32_t *key; /* dimension key column */
  uint64_t rows;
  int32_t n_attr;
  const int32_t *attr[4];
  int32_t n_preds;
  int32_t pred_attr[4], pred_op[4], pred_lo[4], pred_hi[4];
  const int32_t *fact_fk; /* fact column probed into this dimension */
} or_dim;

typedef struct {
  int32_t dim;  /* index into dims, or -1 for a fact column */
  int32_t attr; /* attribute index of that dimension */
  int32_t card; /* codes lie in [0, card) */
  const int32_t *fact_col;
} or_gkey;

typedef struct {
  uint64_t n;
  int32_t n_dims;
  or_dim dims[OR_MAX_DIMS];
  int32_t n_fact_preds;
  or_pred fact_preds[OR_MAX_PREDS];
  int32_t n_group_keys;
  or_gkey group_keys[4];
  int32_t agg_op;
  const int32_t *agg_a, *agg_b;
} or_star_query;
