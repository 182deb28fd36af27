/* Rig bundle adjustment with extrinsic refinement on the B300 (cuSfM,
 * Sec. 4.4 "Extrinsic Refinement").
 *
 * A vehicle carries a rig of cameras; every camera pose is the composition
 * of a vehicle pose (world -> vehicle, one per frame) and an extrinsic
 * (vehicle -> camera, one per rig camera, shared by all frames):
 *     T_c = T_c^v T_v^w.
 * The solver refines vehicle poses, extrinsics and points together by the BA
 * solver's Levenberg-Marquardt iteration on
 *     F = 1/2 sum_k rho(|| pi(K T_c^v T_{v_f}^w X_k) - p_obs ||^2)
 * with left perturbations of both factors (so the composite camera moves by
 * Ad(E) xi_V + xi_E).  Points are eliminated with the BA Schur complement
 * over one "virtual camera" per observed (frame, rig camera) pair; the
 * reduced system over the rig parameters is P^T S P + mu D_rig (P the linear
 * map above, D_rig = diag of P^T U P, Marquardt scaling), held dense
 * (6 (frames + rig cameras) <= 4096) and solved by the one-CTA Cholesky
 * kernel while it fits in shared memory, else by block-Jacobi PCG.
 *
 * Conventions as in ba.h: poses as (qw, qx, qy, qz, tx, ty, tz) of the
 * world -> vehicle and vehicle -> camera maps; one pinhole K shared by all
 * rig cameras.  Fixed frames keep their vehicle pose (fixing one removes the
 * gauge freedom V -> H V, E -> E H^-1 and the rigid world motion); fixed rig
 * cameras keep their extrinsic. */
#ifndef BA_RIG_H
#define BA_RIG_H

#include "ba.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_rig ba_rig;

/* Create a rig solver.  Options read: precision (BA_FP64, or BA_FP32 for
 * the per-observation work, reduced system and its solve, with FP64 cost,
 * gain and damping), solver (BA_SOLVER_AUTO: dense Cholesky while the rig
 * system fits in one CTA's shared memory, else PCG; BA_SOLVER_DENSE;
 * BA_SOLVER_PCG), pcg_tol, pcg_max_iters (the pipelined PCG when its plan
 * keeps the system in shared memory and pcg_tol >= 1e-10), max_lm_iters,
 * huber_delta, mu0, mu_min, device, cuda_stream, use_graph, and
 * prior_abs_weight as lambda_e of the extrinsic prior (Sec. 4.4, the absolute
 * constraint on T_c^v: 1/2 lambda_e ||T_vc - T_vc^init||^2 over the top 3 x 4
 * blocks of the camera-to-vehicle transforms, measured on the extrinsics
 * given to ba_rig_set_problem; 0: off); the others are ignored.  Errors:
 * INVALID_ARG, CUDA. */
ba_status ba_rig_create(const ba_options* opts, ba_rig** out);

/* Load a problem from host arrays (replaces any earlier one):
 *   vehicle_qt [n_frames][7]  initial world -> vehicle poses
 *   extr_qt    [n_rig][7]     initial vehicle -> camera extrinsics
 *   pts        [n_pts][3]     initial points
 *   obs_frame, obs_rc, obs_pt [n_obs]  frame, rig camera and point of each
 *                             observation; obs_uv [n_obs][2] pixels
 *   frame_fixed [n_frames], rc_fixed [n_rig] or NULL
 * Errors: INVALID_ARG (sizes < 1, 6 (n_frames + n_rig) > 4096, an index out
 * of range, a non-finite value, a zero quaternion, a free frame or rig camera
 * without observations, or the BA layout's own checks on the observations: a
 * point with fewer than 2 of them), OOM, CUDA. */
ba_status ba_rig_set_problem(ba_rig* g, int32_t n_frames, int32_t n_rig, int32_t n_pts,
                             int64_t n_obs, const double* vehicle_qt, const double* extr_qt,
                             const double* pts, const int32_t* obs_frame, const int32_t* obs_rc,
                             const int32_t* obs_pt, const double* obs_uv, const ba_intrinsics* K,
                             const uint8_t* frame_fixed, const uint8_t* rc_fixed);

/* Run max_lm_iters LM iterations and wait; the report is ba.h's (rmse_px
 * over the observations).  Errors: STATE, NUMERIC, CUDA. */
ba_status ba_rig_solve(ba_rig* g, ba_report* out);

/* Copy the state to host memory; any pointer may be NULL. */
ba_status ba_rig_get_state(const ba_rig* g, double* vehicle_qt, double* extr_qt, double* pts);

const char* ba_rig_last_error(const ba_rig* g);
void ba_rig_destroy(ba_rig* g);

#ifdef __cplusplus
}
#endif

#endif /* BA_RIG_H */
