/*
 * kpo_internal.h -- oracle planner state (TEST INFRASTRUCTURE ONLY, see
 * kpo.h).  The tree is stored node-major in double precision.
 */
#ifndef KPO_INTERNAL_H
#define KPO_INTERNAL_H

#include "kpo.h"

struct kpo {
  kpo_config cfg;
  int d, N;                /* state and control dimension                 */
  int R;                   /* regions                                     */
  int n_sub_per;           /* sub-regions per region (n')                 */
  int n_sub;               /* R * n'                                      */
  double vol;              /* workspace volume of one region (Eq. 3)      */
  /* free-space-obeying decomposition: a kd-tree whose leaves are the
   * regions; node i: axis (3 = leaf), split, right child (left = i + 1) */
  int kd_n, kd_cap, n_leaves;
  int *kd_axis, *kd_right, *kd_leaf;
  double *kd_split;
  double *leaf_lo, *leaf_hi; /* [n_leaves][3]                             */
  double *region_vol;        /* [R] volume of each region, NULL for grids */
  double *boxes;           /* [nb][6]: lo xyz, hi xyz                     */
  int nb;

  /* tree T, capacity t_e */
  int n;                   /* |T|                                         */
  double *x;               /* [t_e][d]                                    */
  int *parent;
  double *u;               /* [t_e][N] control of the edge into the node  */
  int *steps;              /* integration steps of that edge              */
  int *region, *sub;
  unsigned char *in_ve;    /* 1: V_E, 0: V_O                              */

  /* decomposition R */
  uint64_t *n_valid, *n_invalid;
  uint32_t *cov;
  unsigned char *avail;
  unsigned char *visited;  /* [R * n']                                    */
  double *score, *p_accept;
  uint64_t *thr;           /* Bernoulli threshold: accept iff word < thr  */
  double score_sum;

  int iteration;
  int status;
  int goal_node;

  /* algorithmic work counted during replay (work.c), since the last
   * reset or import; wgrid: the broad-phase grid of the pruned box count */
  kpo_work work;
  int32_t wgrid[3];
  int32_t *wbox;           /* [nb][6] cell range of each box in that grid,
                              NULL until a work grid is set                */
  int32_t *wclear;         /* [cells] clearance of each cell, sixteenths   */

  /* learned proposal */
  double *mlp;           /* parameter vector, NULL when off */
  double mix;
  double *hv_feat, *hv_target;
  int hv_cap, hv_count;
};

/* Builds the kd-tree of the free-space-obeying decomposition from the
 * obstacles (model.c).  Returns 0, or -1 past KPO_FSO_MAX_LEAVES leaves. */
int kpo_build_fso(kpo *o);

/* Work of one sample drawn / one integrator step from x0 to x1 (work.c). */
void kpo_sample_work(kpo *o);
void kpo_step_work(kpo *o, const double *x0, const double *x1);

#endif
