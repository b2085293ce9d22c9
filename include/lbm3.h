/*
 * lbm3.h -- C ABI of the GB300 ternary colour-gradient lattice Boltzmann
 * library (D2Q9).  The method is that of Yu, Liu, Liang & Zhang, "A versatile
 * lattice Boltzmann model for immiscible ternary fluid flows" (arXiv
 * 1808.08555), Sec. 2.  One call of lbm3_step advances every node of a
 * periodic nx x ny grid by one time step: colour gradients (Eq. fd1), the
 * N-phase interfacial force (Eq. 11) applied with Guo's forcing (Eq. 5)
 * inside a BGK collision with harmonic-mean viscosity (Eqs. 1-3, uk1, vis_1,
 * tau), recolouring with the segregation parameters of Eqs. 18-20 (Eq. 6),
 * and streaming of the three colour populations (Eq. 30).
 *
 * Conventions shared by every call
 *  - Colours k = 0, 1, 2 are the paper's r, g, b (fluids 1, 2, 3).
 *    D2Q9 directions i = 0..8: e0 = (0,0), e1 = (1,0), e2 = (0,1),
 *    e3 = (-1,0), e4 = (0,-1), e5 = (1,1), e6 = (-1,1), e7 = (-1,-1),
 *    e8 = (1,-1).
 *  - Node (x, y), 0 <= x < nx, 0 <= y < ny, x fastest; periodic in x and y.
 *  - Host-side arrays are FP64, C order: colour densities rho[3][ny][nx],
 *    populations f[3][9][ny][nx] (post-streaming, i.e. the f_{i,k}(x,t) from
 *    which rho_k = sum_i f_{i,k}).  They always belong to the caller and are
 *    copied.  Where a call takes `on_device`, a non-zero value means the
 *    pointer is a CUDA device pointer of the same layout on the context's
 *    device; the copy is then device-to-device.
 *  - Every call returns an lbm3_status and never aborts the process.  On an
 *    error the text is in lbm3_last_error(ctx).  A NULL context gives
 *    LBM3_EINVAL.
 *  - All device work is ordered on the CUDA stream given to lbm3_create.
 *    lbm3_step is asynchronous; the calls that return host data
 *    synchronise that stream.
 */
#ifndef LBM3_H
#define LBM3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3_ctx lbm3_ctx;

typedef enum {
  LBM3_OK = 0,
  LBM3_EINVAL = 1,   /* bad argument or parameter */
  LBM3_ENOMEM = 2,   /* device allocation failed */
  LBM3_ECUDA = 3,    /* a CUDA call failed; text in lbm3_last_error */
  LBM3_ESTATE = 4,   /* call out of order (e.g. step before init) */
  LBM3_ENUMERIC = 5, /* NaN or Inf found in the state */
  LBM3_ETIMEOUT = 6  /* a bounded in-kernel wait gave up; results invalid */
} lbm3_status;

typedef enum {
  LBM3_FP32 = 0,     /* populations stored as FP32, FP32 arithmetic */
  LBM3_FP16_DEV = 1, /* stored as FP32 rho'_k per node plus FP16 deviations f - w_i rho'_k; FP32 arithmetic */
  LBM3_BF16_DEV = 2, /* the same with BF16 deviations */
  LBM3_REDUCED = 3   /* reduced state, FP32: per node the colour fractions phi_k, the post-collision total
                        distribution f^dagger_i and the recolouring vectors V_k = sum_{l != k} beta_kl
                        (rho_k rho_l / rho) n_kl (18 values instead of 27 populations).  Collision and
                        recolouring use only the total distribution and the colour densities (Eqs. 1, 6),
                        so every population f_{i,k} = phi_k f^dagger_i + w'_i e_i . V_k is rebuilt
                        from its source node in the pull, with the same FP32 operations as the FP32
                        storage: results are bit-identical to LBM3_FP32.  A state set from populations
                        (lbm3_init, lbm3_set_populations) is kept as FP32 populations in an extra
                        buffer until the next step turns it into the reduced state.  Body force only. */
} lbm3_storage;

typedef enum {
  LBM3_BETA_PAPER = 0,    /* Eqs. 18-20: beta^0 [1 + min(35 r g b / rho^3, 1) g(X_kl)] */
  LBM3_BETA_FU = 1,       /* Eq. fu: beta_kl = beta^0 */
  LBM3_BETA_SPENCER = 2,  /* Eq. 16 */
  LBM3_BETA_LECLAIRE = 3  /* Eq. 17 */
} lbm3_beta_form;

typedef enum {
  LBM3_RECOLOR_COSINE = 0, /* Eq. 6 with n_kl.e_i/|e_i| (matches the paper's xi = 1.5831, Sec. 3.1) */
  LBM3_RECOLOR_LITERAL = 1 /* Eq. 6 with n_kl.e_i exactly as printed */
} lbm3_recolor_form;

typedef enum {
  LBM3_FORCE_BODY = 0,         /* the paper's: the force of Eq. 11 through Guo's forcing term (Eq. 5) */
  LBM3_FORCE_PERTURBATION = 1  /* Leclaire et al.'s perturbation operator, Eqs. phi1 / phi_old, with
                                  A_kl = A_lk = 9 sigma_kl / (2 tau_f) and B_0 = -4/27, B_1-4 = 2/27,
                                  B_5-8 = 5/108; u = sum_i f_i e_i / rho.  FP32 storage only. */
} lbm3_force_form;

/* Problem statement (Sec. 2).  Validation in lbm3_create:
 * nx >= 4 and a multiple of 4, ny >= 1, nx*ny < 2^31; tau[k] > 0.5;
 * rho0[k] > 0; sigma_kl > 0; 0 < beta0 <= 1; forms and storage in range;
 * force_form 1 with FP32 storage only; 0 <= normal_delta <= 1. */
typedef struct {
  int32_t nx, ny;
  double tau[3];      /* per-fluid relaxation time; nu_k = (tau_k - 1/2)/3 (Eq. tau) */
  double rho0[3];     /* pure-fluid densities rho_k^0 of Eq. 15 */
  double sigma12, sigma13, sigma23; /* interfacial tensions (Eq. 11) */
  double beta0;       /* reference segregation parameter (0.7 in the paper) */
  int32_t beta_form;  /* lbm3_beta_form */
  int32_t recolor_form; /* lbm3_recolor_form */
  int32_t storage;    /* lbm3_storage */
  int32_t force_form; /* lbm3_force_form (0 for the paper's model) */
  double normal_delta; /* recolouring normal of Eq. 6: n_kl = G_kl / max(|G_kl|, normal_delta phi_k phi_l).
                          0 = the paper's unit normal G_kl/|G_kl| (Sec. 2, after Eq. 11).  A value
                          d > 0 leaves the unit normal wherever |G_kl| >= d phi_k phi_l (across a
                          k-l interface |G_kl| is about 1.26 phi_k phi_l) and takes n_kl continuously
                          to 0 where G_kl vanishes, where the unit normal's direction is decided by
                          rounding.  The Python binding uses 0.1.  In both forms n_kl = 0 where
                          |G_kl| <= 1e-15. */
} lbm3_params;

/* Bytes of ONE population buffer for these parameters, with the row pitch
 * P = max(nx + 8, 136) rounded up to a multiple of 8 (rows carry four ghost
 * columns on each side that hold the periodic wrap): 27 * ny * P * 4 for FP32
 * storage, 27 * ny * P * 2 + 3 * ny * P * 4 for the 16-bit deviation
 * storages, 18 * ny * P * 4 for the reduced state.  Writes *bytes.  No
 * device work. */
lbm3_status lbm3_buffer_bytes(const lbm3_params* p, size_t* bytes);

/* Validate p and create a context bound to the current CUDA device and to
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * context allocates a small reduction scratch area (< 1 MiB).  It allocates
 * the two population buffers itself unless lbm3_bind_buffers is called
 * before the first lbm3_init / lbm3_set_populations.  With a 16-bit deviation
 * storage it also allocates, on the first lbm3_init / lbm3_set_populations /
 * lbm3_populations call, one FP32 buffer (27 * ny * P * 4 bytes) used to
 * convert host data.  *out receives the context (NULL on failure). */
lbm3_status lbm3_create(const lbm3_params* p, void* cuda_stream, lbm3_ctx** out);
/* (The reduced storage allocates the same FP32 buffer, 27 * ny * P * 4
 * bytes, on its first lbm3_init / lbm3_set_populations / lbm3_populations /
 * lbm3_mass / lbm3_phi call; it holds populations set by the caller until
 * the next step, and the expanded populations for reads.) */

/* Use caller-owned device memory for the two population buffers (each at
 * least lbm3_buffer_bytes bytes, 256-byte aligned, distinct).  The caller keeps
 * ownership and must keep both alive until lbm3_destroy.  Only allowed before
 * the state is first set (else LBM3_ESTATE). */
lbm3_status lbm3_bind_buffers(lbm3_ctx* ctx, void* dev_f0, void* dev_f1, size_t bytes_each);

/* Set the state at t = 0 from colour densities rho[3][ny][nx] (FP64; every
 * rho_k >= 0 and rho_r + rho_g + rho_b > 0, else LBM3_EINVAL -- checked on
 * the host for host input, by a device check for device input): populations
 * at rest, f_{i,k} = w_i rho_k (the paper does not state an initialisation;
 * this is the per-colour equilibrium of Eq. 3 with u = 0). */
lbm3_status lbm3_init(lbm3_ctx* ctx, const double* rho, int on_device);

/* Set the state to given post-streaming populations f[3][9][ny][nx] (FP64,
 * rounded to the storage precision).  Resets the step counter to 0.  Used
 * for checkpoint restore and for tests from non-equilibrium states. */
lbm3_status lbm3_set_populations(lbm3_ctx* ctx, const double* f, int on_device);

/* Tuning: rows of the grid each CTA of the fused step kernel marches over.
 * 0 = automatic: one wave of CTAs over the GPU's SMs, with the 124-column
 * strips and a narrower last strip (when 124 does not divide nx) cut into
 * chunks of separately chosen heights.  Otherwise 1..ny, the same height
 * for every strip.  Results are bit-identical for every choice (the
 * arithmetic per node is the same); only speed changes. */
lbm3_status lbm3_set_rows_per_cta(lbm3_ctx* ctx, int32_t rows);

/* Testing hook for the step kernel's bounded waits (FP32 storage with the
 * body force; ignored otherwise).  In the next lbm3_step launch only, which
 * then runs a separate instantiation of the kernel, CTA 0 announces march
 * row `row` (0 = the first halo row of its tile) to its consumers but never
 * copies it.  Its waits
 * then run out after 2 s, the CTA stops without writing its tile, and the
 * next synchronising call (lbm3_mass, lbm3_fields, lbm3_sync) returns
 * LBM3_ETIMEOUT.  That call also clears the error word, so the context stays
 * usable once its state is set again.  -1 cancels; other values below -1
 * are LBM3_EINVAL.  Nothing faults and no wait is unbounded. */
lbm3_status lbm3_debug_stall_row(lbm3_ctx* ctx, int32_t row);

/* Advance n >= 0 time steps (Sec. 2: collision, recolouring, streaming),
 * asynchronously on the context's stream. */
lbm3_status lbm3_step(lbm3_ctx* ctx, int64_t n);

/* Macroscopic fields at the current time t: rho[3][ny][nx] = rho_k
 * (after Eq. 30), ux/uy[ny][nx] from Eq. uk1 (including the F_s/2 term;
 * sum_i f_i e_i / rho with the perturbation-operator force form),
 * p[ny][nx] = rho c_s^2 = rho/3 (the paper gives no pressure formula).
 * Any output pointer may be NULL.  Synchronises the stream when on_device is
 * 0.  Returns LBM3_ETIMEOUT if an earlier kernel reported a timed-out wait. */
lbm3_status lbm3_fields(lbm3_ctx* ctx, double* rho, double* ux, double* uy, double* p, int on_device);

/* Post-streaming populations f[3][9][ny][nx] at time t, widened to FP64. */
lbm3_status lbm3_populations(lbm3_ctx* ctx, double* f, int on_device);

/* FP64 reductions of the current state (synchronises): mass[k] = sum_x rho_k,
 * mom[0..1] = sum_x sum_i f_i e_i (lattice momentum; the F_s/2 term of
 * Eq. uk1 sums to zero on a periodic grid).  Either pointer may be NULL.
 * Returns LBM3_ENUMERIC if a sum is NaN or Inf. */
lbm3_status lbm3_mass(lbm3_ctx* ctx, double* mass, double* mom);

/* Interface diagnostics of the current state, measured in FP64 on the device
 * from the FP64 fields (the paper measures contact angles, Eq. theta_kl, and
 * Laplace jumps, Eqs. laplace and 22, without giving a procedure).
 *  - Interface points of a pair (k, l), m the third colour: on every link
 *    (x, y)-(x+1, y) and (x, y)-(x, y+1) inside the grid (not across the
 *    periodic edges) with phi_k, phi_l > 0 at both ends, where
 *    ln(phi_k / phi_l) changes sign (> 0 at exactly one end) and
 *    phi_m < third_max at both ends, the zero of its linear interpolant
 *    (exact on the tanh profile of Eq. 21).
 *  - circle[q] = (cx, cy, R), q = pairs 12, 13, 23: the algebraic
 *    least-squares circle of the pair's points, min sum (x^2 + y^2 + D x +
 *    E y + F)^2, in grid coordinates (node (x, y) at (x, y)).
 *  - junction[j] = (x, y): the two intersections of circles 12 and 13, each
 *    averaged with the intersections of circles 12/23 and 13/23 nearest to it.
 *  - varphi_junction[j][q]: at junction j each circle's tangent is a line;
 *    with one direction per line chosen so that no half-plane holds all
 *    three, the angle inside fluid m between the interfaces k-m and l-m is
 *    that between their directions, and varphi_kl = 180 - that angle
 *    (degrees; the contact angle of Eq. theta_kl).  varphi = their mean.
 *  - p_bulk[k], n_bulk[k]: mean of p = rho/3 over the n_bulk[k] nodes with
 *    phi_k > bulk_min (NaN if none): p_bulk[k] - p_bulk[l] is the Laplace
 *    jump across a k-l interface.
 *  - flags: bit 0 a pair has fewer than 3 points (its circle and every angle
 *    are NaN), bit 1 circles 12 and 13 do not meet, bit 2 the interfaces do
 *    not surround a junction (angles NaN in either case).
 * Written for a droplet that does not cross the periodic edges.  Uses the
 * idle population buffer as FP64 staging and, on its first call, allocates
 * 271 KB of device scratch.  Synchronises the stream.  0 < third_max <= 1,
 * 0 < bulk_min < 1, else LBM3_EINVAL. */
typedef struct {
  double varphi[3];
  double varphi_junction[2][3];
  double junction[2][2];
  double circle[3][3];
  double points[3];
  double p_bulk[3];
  double n_bulk[3];
  int32_t flags;
} lbm3_interfaces;
lbm3_status lbm3_interface_diagnostics(lbm3_ctx* ctx, double third_max, double bulk_min, lbm3_interfaces* out);

/* Replace the physical parameters (tau, rho0, sigma_kl, beta0, beta_form,
 * recolor_form) of a context; nx, ny and storage must stay the same
 * (LBM3_EINVAL otherwise).  The state is kept; a recorded run (below) is
 * dropped. */
lbm3_status lbm3_set_params(lbm3_ctx* ctx, const lbm3_params* p);

/* Colour fractions phi_k = rho_k / rho (after Eq. 30) at the current time,
 * phi[3][ny][nx] in FP64 (FP32 and reduced storage only, LBM3_EINVAL otherwise).
 * Synchronises the stream when on_device is 0. */
lbm3_status lbm3_phi(lbm3_ctx* ctx, double* phi, int on_device);

/* ------------------------------------------------------------------------
 * Reverse mode.  Gradients of a scalar loss J(phi(t_end)) of the final colour
 * fractions with respect to the initial state and to the interfacial
 * tensions sigma_kl, through every step of Sec. 2 (the force of Eq. 11 and
 * the segregation parameters of Eqs. 16-20 both depend on sigma_kl).  The
 * paper defines no adjoint; this is the exact transpose of the linearised
 * step, taken in FP32 with the scalar gradients summed in FP64.
 *
 * lbm3_tape_forward advances nsteps >= 1 steps from the current state like
 * lbm3_step and records the run: it keeps a copy of the state every
 * checkpoint_every >= 1 steps (ceil(nsteps / checkpoint_every) states) and
 * allocates room for checkpoint_every - 1 more, into which lbm3_tape_backward
 * recomputes one segment at a time.  State memory: lbm3_buffer_bytes() each,
 * so checkpoint_every near sqrt(nsteps) minimises it and checkpoint_every = 1
 * stores every state and recomputes nothing.  FP32 storage only
 * and the paper's force form (LBM3_EINVAL otherwise), LBM3_ENOMEM if the
 * states do not fit.
 *
 * lbm3_tape_backward takes dJ/dphi[3][ny][nx] (FP64, host or device) at the
 * end of the recorded run and writes, for any non-NULL output:
 *   dpop0[3][9][ny][nx]  dJ/df_{i,k}(x, 0) of the post-streaming populations
 *                        the run started from (FP64, the layout of
 *                        lbm3_set_populations),
 *   drho0[3][ny][nx]     dJ/drho_k(x, 0) for a start from lbm3_init (rest
 *                        equilibrium f_{i,k} = w_i rho_k), i.e.
 *                        sum_i w_i dpop0_{i,k}(x),
 *   dsigma[3]            dJ/d(sigma_12, sigma_13, sigma_23) (host memory).
 * dpop0 and drho0 are host arrays when out_on_device is 0 (the call then
 * synchronises) and device arrays otherwise.  LBM3_ESTATE without a recorded
 * run (lbm3_init, lbm3_set_populations, lbm3_step and lbm3_set_params drop
 * it); LBM3_ENUMERIC if a gradient is not finite.  The context's state is
 * left at the end of the run. */
lbm3_status lbm3_tape_forward(lbm3_ctx* ctx, int64_t nsteps, int32_t checkpoint_every);
lbm3_status lbm3_tape_backward(lbm3_ctx* ctx, const double* dphi, int dphi_on_device, double* dpop0, double* drho0,
                               int out_on_device, double* dsigma);

/* ------------------------------------------------------------------------
 * Batches: many independent simulations advanced together (a parameter or
 * morphology sweep).  Each instance has its own grid size and parameters;
 * one kernel launch per step covers every tile of every instance, and the
 * steps are replayed from a captured two-step CUDA graph.  Per-instance
 * results are bit-identical to running the same instance alone (same
 * arithmetic per node).  The paper runs its cases one at a time; batching is
 * a property of this library, not of the method.
 * ------------------------------------------------------------------------ */
typedef struct lbm3_batch lbm3_batch;

/* Create `count` instances from params[0..count-1] (each validated as in
 * lbm3_create; every instance with the body force and the same storage,
 * LBM3_FP32 or LBM3_REDUCED, else LBM3_EINVAL) on the current device and
 * `cuda_stream`.  All state buffers (and, for the reduced state, each
 * instance's FP32 population buffer) are allocated here.  With the reduced
 * state, the first step after instances were set (lbm3_batch_init /
 * _set_populations) reads their populations; if only some were set, that
 * step runs as two launches (the set instances, the others).  rows_per_cta: rows per work item (0 =
 * automatic: the tile height whose largest-first assignment of work items to
 * the GPU's resident CTA slots gives the shortest estimated step).
 * *out receives the batch (NULL on failure). */
lbm3_status lbm3_batch_create(const lbm3_params* params, int32_t count, void* cuda_stream, int32_t rows_per_cta,
                              lbm3_batch** out);
/* Empirical tile-height tuning of a batch.  Times `candidates` (1..16) tile
 * heights -- the best ranked by the batch's makespan model (largest-first
 * assignment of the work items to the GPU's resident CTA slots), plus 64 and
 * 128 rows when not among them -- with one warm-up and `steps` >= 1 timed
 * launches each (CUDA events on the batch's stream), on the current state:
 * every timed launch reads the current state and writes the idle buffers,
 * so neither the state nor lbm3_batch_time changes.  Keeps the fastest
 * height for lbm3_batch_step.  *rows and *ms_per_step (either may be NULL)
 * receive the winner; table (may be NULL) receives (candidates + 2) pairs
 * (rows, ms per launch), unused pairs zero.  Every instance must be
 * initialised, and with the reduced state have stepped since it was last set
 * (else LBM3_ESTATE).  Synchronises the stream.  Results of
 * later steps do not depend on the height (same arithmetic per node). */
lbm3_status lbm3_batch_autotune(lbm3_batch* b, int32_t candidates, int32_t steps, int32_t* rows,
                                double* ms_per_step, double* table);
/* Number of instances; number of CTA work items of one step. */
int32_t lbm3_batch_count(const lbm3_batch* b);
int32_t lbm3_batch_work_items(const lbm3_batch* b);
/* Per-instance state set-up and read-out, as the lbm3_* calls of the same
 * name for instance i (0 <= i < count). */
lbm3_status lbm3_batch_init(lbm3_batch* b, int32_t i, const double* rho, int on_device);
lbm3_status lbm3_batch_set_populations(lbm3_batch* b, int32_t i, const double* f, int on_device);
lbm3_status lbm3_batch_fields(lbm3_batch* b, int32_t i, double* rho, double* ux, double* uy, double* p,
                              int on_device);
lbm3_status lbm3_batch_populations(lbm3_batch* b, int32_t i, double* f, int on_device);
lbm3_status lbm3_batch_mass(lbm3_batch* b, int32_t i, double* mass, double* mom);
/* Advance every instance by n >= 0 steps (asynchronous; every instance must
 * have been initialised, else LBM3_ESTATE). */
lbm3_status lbm3_batch_step(lbm3_batch* b, int64_t n);
lbm3_status lbm3_batch_sync(lbm3_batch* b);
int64_t lbm3_batch_time(const lbm3_batch* b);
lbm3_status lbm3_batch_destroy(lbm3_batch* b);
const char* lbm3_batch_last_error(const lbm3_batch* b);

/* Allocation-free FP64 mass/momentum reduction, for callers that cannot
 * call cudaMalloc (all their device memory is owned by their own pool or
 * allocator, or they run under a fixed device-memory budget).  The paper has
 * no counterpart: this is a service of the library, not part of the method.
 *
 * dev_f: device array of FP32 populations on the current CUDA device, in
 * the plain layout of the host-side calls: unpadded, [3][9][ny][nx] (plane
 * k*9 + i holds colour k, direction i; rows of exactly nx values).  This is
 * NOT the layout of the library's own population buffers (padded rows with
 * ghost columns, planes grouped by direction), which lbm3_mass reduces
 * instead.  Whether the values are pre- or post-streaming does not matter:
 * the sums over all nodes are the same.  dev_out: device array of 5 doubles receiving
 * (mass_r, mass_g, mass_b, mom_x, mom_y) as in lbm3_mass.  Work is enqueued on
 * `cuda_stream` (a cudaStream_t of the current device; NULL = legacy default
 * stream); the call does not synchronise.
 *
 * Scratch: block partial sums live in a file-scope device array of 1024 x 5
 * doubles (40 KiB) that every GPU loading the library holds until exit, so
 * nx*ny may be at most 16,777,216 (1024 blocks x 16384 nodes; e.g. 4096^2).
 * Larger grids, NULL pointers or non-positive sizes return LBM3_EINVAL; CUDA
 * failures return LBM3_ECUDA.  The first call on each device looks the
 * array's device address up (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  No memory is allocated or
 * freed.  All calls share the one array: calls whose work overlaps on the GPU
 * (other streams, other threads) race on it and must be serialised by the
 * caller.  Each call overwrites the partials it reads, so no clearing is
 * needed between calls. */
lbm3_status lbm3_mass_noalloc(const float* dev_f, int32_t nx, int32_t ny, void* cuda_stream, double* dev_out);

/* ------------------------------------------------------------------------
 * N fluids (2 <= nfluids <= 6).  The paper writes the interfacial force
 * (Eq. 11) and the recolouring (Eq. 6) for any number of fluids and simulates
 * three.  This context runs the same step (Eq. fd1 gradients, Eq. 11 force
 * through Guo's term, BGK with the harmonic-mean viscosity, recolouring,
 * streaming) for N fluids, as three kernels per step over global-memory
 * intermediates (a first path: not the fused, TMA-fed kernel of lbm3_step).
 * beta_kl for N fluids, which the paper does not give beyond three:
 *   beta_kl = beta0 [1 + sum_{m != k, l} min(35 rho_k rho_l rho_m / rho^3, 1) g(X_kl^m)]
 * with X_kl^m of Eq. 18 for the third fluid m and g of Eq. 20: Eq. 19
 * exactly for N = 3, one junction term per third fluid beyond (beta_form 1:
 * the constant beta0 of Eq. fu).  Arrays: sigma[nfluids][nfluids] symmetric
 * with a zero diagonal and positive entries off it; tau, rho0 [nfluids];
 * host densities rho[N][ny][nx] and populations f[N][9][ny][nx] (FP64,
 * post-streaming) as for the three-fluid calls; the state is FP32.  Any
 * invalid parameter gives LBM3_EINVAL from lbm3n_create.  The context
 * allocates its two population buffers, the intermediates
 * ((14 + v + 2 N) nx ny floats, v = 2 for N = 2, 4 for N = 3, 4 and 8
 * for N = 5, 6) and an FP64 staging area.
 * storage LBM3_REDUCED keeps, per node, the colour fractions phi_k, the
 * recolouring vectors V_k and the post-collision total distribution
 * f^dagger_i (3 N + 9 values instead of 9 N, in the same buffers), as
 * LBM3_REDUCED does for lbm3_ctx: results are bit-identical to LBM3_FP32; a
 * state set from populations is held as populations until the next step, and
 * lbm3n_populations / lbm3n_mass expand the reduced state into the idle
 * buffer first. */
typedef struct lbm3n_ctx lbm3n_ctx;
typedef struct {
  int32_t nx, ny, nfluids;
  const double* tau;    /* [nfluids], each > 0.5 */
  const double* rho0;   /* [nfluids], each > 0 (Eq. 15) */
  const double* sigma;  /* [nfluids][nfluids] */
  double beta0;         /* (0, 1] */
  int32_t beta_form;    /* 0: the N-fluid form above; 1: Eq. fu */
  int32_t recolor_form; /* as lbm3_recolor_form */
  double normal_delta;  /* as lbm3_params.normal_delta */
  int32_t storage;      /* LBM3_FP32 or LBM3_REDUCED (below) */
} lbm3n_params;
lbm3_status lbm3n_create(const lbm3n_params* p, void* cuda_stream, lbm3n_ctx** out);
/* rest equilibrium per colour from host densities (rho_k >= 0) */
lbm3_status lbm3n_init(lbm3n_ctx* ctx, const double* rho, int on_device);
lbm3_status lbm3n_set_populations(lbm3n_ctx* ctx, const double* f, int on_device);
lbm3_status lbm3n_step(lbm3n_ctx* ctx, int64_t n);  /* asynchronous */
lbm3_status lbm3n_populations(lbm3n_ctx* ctx, double* f, int on_device);  /* synchronises */
/* FP64 per-fluid mass[nfluids] and lattice momentum mom[2] (synchronises) */
lbm3_status lbm3n_mass(lbm3n_ctx* ctx, double* mass, double* mom);
/* Observables of the current state, as lbm3_fields: rho_k [N][ny][nx], ux,
 * uy [ny][nx] = (sum_i f_i e_i + F/2) / rho with the force of Eq. 11,
 * p = rho / 3; FP64 host pointers or, with on_device, device pointers; any
 * may be NULL.  Synchronises. */
lbm3_status lbm3n_fields(lbm3n_ctx* ctx, double* rho, double* ux, double* uy, double* p, int on_device);
lbm3_status lbm3n_destroy(lbm3n_ctx* ctx);
const char* lbm3n_last_error(const lbm3n_ctx* ctx);

/* ------------------------------------------------------------------------
 * N fluids on the D3Q19 lattice (2 <= nfluids <= 4).  The paper writes the
 * model in vector form (Eq. fd1, the interfacial force of Eq. 11, the
 * recolouring of Eq. 6) and simulates two dimensions on D2Q9.  This context
 * runs the same step in three dimensions: Eq. fd1 gradients with the D3Q19
 * weights (1/3 rest, 1/18 axis, 1/36 edge diagonals, c_s^2 = 1/3), the 3x3
 * tension tensor of Eq. 11, Guo's forcing, BGK with the harmonic-mean
 * viscosity, recolouring (w'_i = w_i / |e_i|, or w_i with recolor_form 1),
 * pull streaming; beta_kl as for lbm3n.  Three kernels per step over
 * global-memory intermediates (a first path).  Directions, opposite pairs
 * adjacent:
 *   0 (0,0,0)  1 (1,0,0)  2 (-1,0,0)  3 (0,1,0)  4 (0,-1,0)  5 (0,0,1)
 *   6 (0,0,-1)  7 (1,1,0)  8 (-1,-1,0)  9 (1,-1,0)  10 (-1,1,0)  11 (1,0,1)
 *   12 (-1,0,-1)  13 (1,0,-1)  14 (-1,0,1)  15 (0,1,1)  16 (0,-1,-1)
 *   17 (0,1,-1)  18 (0,-1,1)
 * Arrays: sigma[nfluids][nfluids] symmetric with a zero diagonal and
 * positive entries off it; tau, rho0 [nfluids]; host densities
 * rho[N][nz][ny][nx] and populations f[N][19][nz][ny][nx] (FP64,
 * post-streaming: the populations whose densities are the state at time t);
 * the state is FP32, periodic in all three directions.  ny, nz <= 65535.
 * Any invalid parameter gives LBM3_EINVAL from lbm3d_create.  The context
 * allocates its two population buffers (19 N nx ny nz floats each), the
 * intermediates ((4 + 25 + 3 N (N - 1) / 2) nx ny nz floats for N <= 3,
 * 4 more per node for N = 4) and an FP64 staging area of one population
 * state.
 * storage LBM3_REDUCED keeps, per node, the colour fractions phi_k, the
 * post-collision total distribution f^dagger_i and the recolouring vectors
 * V_k (19 + 4 N floats instead of 19 N, in the same buffers), as LBM3_REDUCED
 * does for lbm3_ctx; every population is rebuilt from its source node with
 * the FP32 operations of the population form, so results are bit-identical
 * to LBM3_FP32.  A state set by lbm3d_init / lbm3d_set_populations is held as
 * populations until the next step; lbm3d_populations and lbm3d_mass expand
 * the reduced state into the idle buffer first. */
typedef struct lbm3d_ctx lbm3d_ctx;
typedef struct {
  int32_t nx, ny, nz, nfluids;
  const double* tau;    /* [nfluids], each > 0.5 */
  const double* rho0;   /* [nfluids], each > 0 (Eq. 15) */
  const double* sigma;  /* [nfluids][nfluids] */
  double beta0;         /* (0, 1] */
  int32_t beta_form;    /* 0: Eq. 19 with one junction term per third fluid; 1: Eq. fu */
  int32_t recolor_form; /* as lbm3_recolor_form */
  double normal_delta;  /* as lbm3_params.normal_delta */
  int32_t storage;      /* LBM3_FP32 or LBM3_REDUCED (below) */
} lbm3d_params;
lbm3_status lbm3d_create(const lbm3d_params* p, void* cuda_stream, lbm3d_ctx** out);
/* rest equilibrium per colour from host densities (rho_k >= 0) */
lbm3_status lbm3d_init(lbm3d_ctx* ctx, const double* rho, int on_device);
lbm3_status lbm3d_set_populations(lbm3d_ctx* ctx, const double* f, int on_device);
lbm3_status lbm3d_step(lbm3d_ctx* ctx, int64_t n);  /* asynchronous */
lbm3_status lbm3d_populations(lbm3d_ctx* ctx, double* f, int on_device);  /* synchronises */
/* FP64 per-fluid mass[nfluids] and lattice momentum mom[3] (synchronises) */
lbm3_status lbm3d_mass(lbm3d_ctx* ctx, double* mass, double* mom);
/* Observables of the current state (Eq. uk1, as lbm3_fields): rho_k
 * [N][nz][ny][nx], u [3][nz][ny][nx] = (sum_i f_i e_i + F/2) / rho with the
 * interfacial force F of Eq. 11, p [nz][ny][nx] = rho / 3, FP64; host pointers
 * or, with on_device, device pointers; any of the three may be NULL.
 * Synchronises. */
lbm3_status lbm3d_fields(lbm3d_ctx* ctx, double* rho, double* u, double* p, int on_device);
lbm3_status lbm3d_destroy(lbm3d_ctx* ctx);
const char* lbm3d_last_error(const lbm3d_ctx* ctx);

/* Wait for the context's stream and report device-side errors (timed-out
 * waits) recorded since the last check. */
lbm3_status lbm3_sync(lbm3_ctx* ctx);

/* Number of steps taken since the last init / set_populations. */
int64_t lbm3_time(const lbm3_ctx* ctx);

/* Free the context and everything it allocated (bound buffers are not
 * freed).  Synchronises its stream first.  NULL is accepted. */
lbm3_status lbm3_destroy(lbm3_ctx* ctx);

/* Text of the last error on this context ("" if none); a static string for
 * ctx == NULL.  Valid until the next call on the context. */
const char* lbm3_last_error(const lbm3_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM3_H */
