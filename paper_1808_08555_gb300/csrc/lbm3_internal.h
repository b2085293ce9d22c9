// Internal declarations shared by the CUDA translation units of liblbm3.
// Nothing here is part of the public C ABI (see include/lbm3.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lbm3 {

// ---------------------------------------------------------------- lattice
// D2Q9 (arXiv 1808.08555, Sec. 2 after Eq. 3): e0 = (0,0), e1 = (1,0),
// e2 = (0,1), e3 = (-1,0), e4 = (0,-1), e5 = (1,1), e6 = (-1,1), e7 = (-1,-1),
// e8 = (1,-1); w0 = 4/9, w1-4 = 1/9, w5-8 = 1/36.
__host__ __device__ constexpr int ex(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// FP32 weights chosen so that w0 + 4 w1 + 4 w5 = 1 holds exactly: w1 and
// w5 = w1/4 are one ulp below 1/9 and 1/36, w0 one ulp above 4/9.  With the
// nearest-float weights the sum is 1 + 7.5e-9, which makes the collision
// create mass at a steady ~1e-8 relative per step.
__host__ __device__ constexpr float wt(int i) {
  return i == 0 ? 0x1.c71c74p-2f : (i < 5 ? 0x1.c71c70p-4f : 0x1.c71c70p-6f);
}

// ------------------------------------------------------------ HBM layout
// Populations are stored as 27 planes of ny rows with a padded pitch
// P = max(nx + 8, 132): column xp = x + 4 holds node x, and the four ghost
// columns on each side hold copies of the opposite edge (periodic wrap), so
// that every strip's halo window is one contiguous, in-bounds span of a row.  Planes are
// ordered by the y-component of their direction so that the nine planes a
// pulled row needs from one source row are consecutive:
//   group 0: e_y = +1 {2, 5, 6}; group 1: e_y = 0 {0, 1, 3}; group 2: e_y = -1 {4, 7, 8}
//   plane(k, i) = 9 * group(i) + 3 * k + position of i in its group.
constexpr int kGhost = 4;
__host__ __device__ constexpr int dir_group(int i) { return ey(i) > 0 ? 0 : (ey(i) == 0 ? 1 : 2); }
__host__ __device__ constexpr int dir_pos(int i) {
  return (i == 2 || i == 0 || i == 4) ? 0 : ((i == 5 || i == 1 || i == 7) ? 1 : 2);
}
__host__ __device__ constexpr int plane_of(int k, int i) { return 9 * dir_group(i) + 3 * k + dir_pos(i); }
// at least one full TMA box wide (kPW, defined below): narrow grids get unused
// columns after the right ghosts so that every box row has the same pitch
constexpr int kBoxCols = 132;  // = kPW below
__host__ __device__ constexpr int pitch_of(int nx) {
  return nx + 2 * kGhost > kBoxCols ? nx + 2 * kGhost : kBoxCols;
}

// ------------------------------------------------------- fused step tiling
// One CTA owns a strip of up to kTX columns and a run of rows; it marches up
// the rows two at a time with a 3-stage pipeline (densities -> tension tensor
// -> force, collision, recolouring) fed by bulk async copies of pulled rows.
// 124 columns: the D stage then has exactly 2 x 128 = 256 nodes per pair of
// rows, one per consumer thread (T: 252, C: 248), so no warp does a second pass
constexpr int kTX = 124;          // max strip width (columns)
constexpr int kPW = kTX + 8;      // population row window: x0-4 .. x0+w+4 (one TMA box row)
static_assert(kPW == kBoxCols, "pitch_of() must cover one TMA box");
constexpr int kGroupFloats = (9 * kPW + 31) / 32 * 32;  // 9 planes x kPW, padded to a 128-byte multiple
constexpr int kDW = kTX + 4;      // density/phi window:     x0-2 .. x0+w+2
constexpr int kTW = kTX + 2;      // tension-tensor window:  x0-1 .. x0+w+1
constexpr int kSlots = 6;         // population ring depth (rows)
constexpr int kConsumers = 256;   // 8 compute warps: one C-stage node each per pair of rows
constexpr int kThreads = kConsumers + 32;  // + 1 copy-issuing warp

struct StepArgs {
  const float* fin;   // stored post-collision populations at t-1, [27][ny][P] (padded layout)
  float* fout;        // written at t (MODE_STEP), same layout
  int nx, ny;
  int pitch;          // P = nx + 8
  int boxw;           // TMA box width in columns: min(kPW, P)
  int nstrips;        // ceil(nx / kTX)
  int rows_per_cta;   // H
  float inv_nu[3];    // 1/nu_k, nu_k = (tau_k - 1/2)/3 (so 1/nu = sum_k phi_k/nu_k)
  float cpair[3];     // 1e6 / (rho0_k rho0_l) for pairs (12, 13, 23)
  float sigma[3];     // sigma_12, sigma_13, sigma_23
  float beta0;
  float beta_A;       // beta_kl = beta0 (1 + min(beta_A * r g b / rho^3, 1) * beta_h[kl])
  float beta_h[3];
  float wrec[9];      // recolouring weight per direction: w_i / |e_i|^p
  unsigned int* err;  // device error word (bit 0: a bounded wait timed out)
  // MODE_FIELDS outputs (FP64, [3][N] and [N]); NULL entries are skipped
  double* out_rho;
  double* out_ux;
  double* out_uy;
  double* out_p;
};

enum { MODE_STEP = 0, MODE_FIELDS = 1 };

size_t step_smem_bytes();
cudaError_t step_configure();  // sets the dynamic shared memory attribute
// tmap: a CUtensorMap (128 bytes) describing a.fin as a 3D tensor
// (P, ny, 27) of FP32 with box (boxw, 1, 9)
cudaError_t launch_step(const StepArgs& a, const void* tmap, int grid, int mode, cudaStream_t s);
// encode that tensor map for a population buffer (uses the driver's encoder)
cudaError_t encode_population_map(void* tmap, const float* buf, int nx, int ny);
int step_occupancy(int* blocks_per_sm);

// ------------------------------------------------------------- aux kernels
cudaError_t launch_init_from_rho(const double* rho, float* f, int nx, int ny, cudaStream_t s);
cudaError_t launch_set_planes(const double* fpost, float* f, int nx, int ny, int plane0, int nplanes,
                              cudaStream_t s);
cudaError_t launch_get_planes(const float* f, double* fpost, int nx, int ny, int plane0, int nplanes,
                              cudaStream_t s);
cudaError_t launch_check_rho(const double* rho, int n, unsigned int* bad, cudaStream_t s);
// FP64 reductions: partial[blocks][5] then out[5] = (mass_r, mass_g, mass_b, mom_x, mom_y)
int reduce_blocks(int N);
// plain [27][ny][nx] array, plane = k*9 + i (the allocation-free entry point's input)
cudaError_t launch_reduce(const float* f, int N, double* partial, int blocks, double* out, cudaStream_t s);
// the library's padded, group-ordered layout
cudaError_t launch_reduce_padded(const float* f, int nx, int ny, double* partial, int blocks, double* out,
                                 cudaStream_t s);

}  // namespace lbm3
