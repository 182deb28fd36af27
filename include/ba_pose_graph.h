/* Pose-graph optimisation on the B300 (cuSfM, Sec. 4.2 "Pose Graph
 * Optimization"): the LM / block-Jacobi PCG machinery of the BA solver run on
 * a camera-only graph.
 *
 * Nodes are camera poses (world -> camera, the same 7-number convention as
 * ba.h).  Every edge (i, j) is a relative-pose constraint; the three kinds of
 * the paper -- sequential constraints from the initial trajectory (Eq. seq),
 * loop closures from stereo relative-pose estimation and extrinsic
 * constraints between the cameras of one rig (Eq. extrinsic) -- share its
 * form.  An edge carries the measured pose M_e of frame i in frame j and a
 * weight w_e >= 0 (the weight matrix Omega_e = w_e I of the paper's
 * objective).  The solver minimises
 *     F = 1/2 sum_e w_e || T_cw,j T_wc,i - M_e ||_F^2
 * over the free nodes (top 3 x 4 blocks; the bottom rows agree), by the BA
 * solver's Levenberg-Marquardt iteration with the same left perturbation
 * T_cw <- Exp(xi) T_cw, Marquardt damping D = diag(A) (clamped to >= 1e-12)
 * and gain-ratio rule.  Fixed nodes keep their pose; a graph without a fixed
 * node has a 6-DoF gauge freedom that only the damping holds.
 *
 * Errors are reported as in ba.h (ba_status; ba_pg_last_error for text). */
#ifndef BA_POSE_GRAPH_H
#define BA_POSE_GRAPH_H

#include "ba.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_pose_graph ba_pose_graph;

/* Create a pose-graph solver.  Options read: precision (BA_FP64: every step
 * in FP64; BA_FP32: the damped system and the PCG in FP32, everything else
 * FP64), solver and dense_max_dim (dense Cholesky of the 6n x 6n system or
 * block-Jacobi PCG, as in ba.h), max_lm_iters, pcg_tol, pcg_max_iters,
 * pcg_variant (0: auto, the pipelined PCG when the system fits in shared
 * memory and pcg_tol >= 1e-10, else the standard one; 1: standard; 2:
 * pipelined, whose attainable relative residual on ill-conditioned graphs
 * can stay above 1e-9), mu0, mu_min, device, cuda_stream, use_graph, alloc /
 * free_fn / alloc_ctx; the others are ignored.  Errors: INVALID_ARG, CUDA. */
ba_status ba_pg_create(const ba_options* opts, ba_pose_graph** out);

/* Load a graph (replaces any earlier one) and build its device layout: the
 * block pattern of the damped system (a diagonal block per node and one
 * off-diagonal block pair per pair of free nodes joined by an edge), each
 * node's incident edges and each node pair's edges.
 *   node_qt   [n_nodes][7]  initial poses (qw, qx, qy, qz, tx, ty, tz)
 *   edge_ij   [n_edges][2]  nodes (i, j) of each edge, i != j
 *   edge_qt   [n_edges][7]  measured pose of frame i in frame j
 *   edge_w    [n_edges]     weights, finite and >= 0
 *   node_fixed [n_nodes] or NULL: nonzero = pose held fixed
 * mem_kind: BA_MEM_HOST or BA_MEM_DEVICE for all five arrays (device arrays
 * are copied to the host for the layout).  Duplicate edges are allowed.
 * Errors: INVALID_ARG when n_nodes < 1, n_edges < 0, an index is out of
 * range or i == j, a value is not finite, a quaternion is zero, a weight is
 * negative, or a free node has no edge of positive weight; OOM; CUDA. */
ba_status ba_pg_set_graph(ba_pose_graph* g, int32_t n_nodes, const double* node_qt,
                          int32_t n_edges, const int32_t* edge_ij, const double* edge_qt,
                          const double* edge_w, const uint8_t* node_fixed, int mem_kind);

/* Run max_lm_iters LM iterations from the current state and wait for them;
 * a second call continues from the state the first left.  The report is
 * ba.h's: cost[], accepted[], mu[], pcg_iters[], pcg_rel_residual[], gain[],
 * solve_ms, setup_ms and n_kernels as there; rmse_px holds the root mean
 * square of the edge residual entries, sqrt(sum_e ||r_e||^2 / (12 E)), at
 * the final state, and n_valid_obs the number of edges.  out may be NULL.
 * Errors: STATE (no graph), TIMEOUT (a PCG grid barrier gave up), NUMERIC
 * (non-finite cost), CUDA. */
ba_status ba_pg_solve(ba_pose_graph* g, ba_report* out);

/* Copy the current node poses out ([n_nodes][7], qw >= 0) to host or device
 * memory.  Errors: STATE, INVALID_ARG, CUDA. */
ba_status ba_pg_get_state(const ba_pose_graph* g, double* node_qt_out, int mem_kind);

/* Text of the last error on g (or of the last failed ba_pg_create when g is
 * NULL).  Valid until the next call on g. */
const char* ba_pg_last_error(const ba_pose_graph* g);

/* Release every device buffer of g; g may be NULL. */
void ba_pg_destroy(ba_pose_graph* g);

#ifdef __cplusplus
}
#endif

#endif /* BA_POSE_GRAPH_H */
