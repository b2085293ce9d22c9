// Internal declarations shared by the CUDA translation units of liblbm3.
// Nothing here is part of the public C ABI (see include/lbm3.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/lbm3.h"

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
// that every strip's halo window is one contiguous span of a row.  Planes are
// ordered by the y-component of their direction so that the nine planes a
// pulled row needs from one source row are consecutive:
//   group 0: e_y = +1 {2, 5, 6}; group 1: e_y = 0 {0, 1, 3}; group 2: e_y = -1 {4, 7, 8}
//   plane(k, i) = 9 * group(i) + 3 * k + position of i in its group.
constexpr int kGhost = 4;
// storage of the state between steps.  ST_RED is the reduced state (below);
// ST_F2R is a step that reads FP32 populations and writes the reduced state
// (the first step after the state was set from populations).
enum { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2, ST_RED = 3, ST_F2R = 4 };
__host__ __device__ constexpr int st_in(int st) { return st == ST_F2R ? ST_FP32 : st; }
__host__ __device__ constexpr int st_out(int st) { return st == ST_F2R ? ST_RED : st; }
__host__ __device__ constexpr int dir_group(int i) { return ey(i) > 0 ? 0 : (ey(i) == 0 ? 1 : 2); }
__host__ __device__ constexpr int dir_pos(int i) {
  return (i == 2 || i == 0 || i == 4) ? 0 : ((i == 5 || i == 1 || i == 7) ? 1 : 2);
}
__host__ __device__ constexpr int plane_of(int k, int i) { return 9 * dir_group(i) + 3 * k + dir_pos(i); }
// at least one full TMA box wide (kPW, defined below): narrow grids get unused
// columns after the right ghosts so that every box row has the same pitch
constexpr int kBoxCols = 132;     // = kPW below: FP32 box width (also the rho' box of 16-bit storage)
constexpr int kDevBoxCols = 136;  // 16-bit box width: a multiple of 8 columns (16 bytes)
// Row pitch shared by every storage: at least one 16-bit box wide and a
// multiple of 8 columns, so that 16-bit rows start on 16-byte boundaries.
__host__ __device__ constexpr int pitch_of(int nx) {
  return ((nx + 2 * kGhost > kDevBoxCols ? nx + 2 * kGhost : kDevBoxCols) + 7) / 8 * 8;
}

// 16-bit deviation storage: a stored population f is kept as
// w_i rho'_k + d with d rounded to FP16 or BF16 (round to nearest even) and
// rho'_k chosen per node so that the 9 rounded values of a colour still sum
// to its mass (see the encode step of the fused kernel).
template <int ST>
__device__ __forceinline__ unsigned short enc16(float v) {
  if (ST == ST_FP16) return __half_as_ushort(__float2half_rn(v));
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <int ST>
__device__ __forceinline__ float dec16(unsigned short b) {
  if (ST == ST_FP16) return __half2float(__ushort_as_half(b));
  return __uint_as_float(static_cast<unsigned int>(b) << 16);
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
// 16-bit storage slot: three boxes of 9 deviation planes x kDevBoxCols (2 bytes)
// and three boxes of the 3 FP32 rho' planes x kPW, each on a 128-byte boundary
constexpr int kDevGroupHalfs = (9 * kDevBoxCols + 63) / 64 * 64;
constexpr int kRhoGroupFloats = (3 * kPW + 31) / 32 * 32;
static_assert(3 * kDevGroupHalfs * 2 + 3 * kRhoGroupFloats * 4 <= 3 * kGroupFloats * 4,
              "a 16-bit slot must fit in an FP32 slot");
// Reduced state (collision and recolouring use only the total distribution
// and the colour densities, Eqs. 1 and 6): per node the colour fractions
// phi_k, the post-collision totals f^dagger_i and the recolouring vectors
// V_k = sum_{l != k} beta_kl (rho_k rho_l / rho) n_kl, from which a pulled
// population is f_{i,k}(x) = phi_k f^dagger_i + w'_i e_i . V_k at x - e_i.
// HBM: three float4 planes A = (phi_1, phi_2, phi_3, fd_0),
// X = (V_1x, V_2x, V_3x, fd_1), Y = (V_1y, V_2y, V_3y, fd_2), then six float
// planes fd_3 .. fd_8, in the padded row layout (72 bytes per padded node).
// A ring slot holds one source row: the three vector planes (one 4D TMA box)
// then the six scalar planes (one 3D box), each 128-byte aligned.
constexpr int kRedVecFloats = (3 * kPW * 4 + 31) / 32 * 32;
constexpr int kRedSclFloats = (6 * kPW + 31) / 32 * 32;
constexpr int kRedSlotFloats = kRedVecFloats + kRedSclFloats;
constexpr int kRedSlots = 6;  // a march-row pair needs 4 source rows; 2 more are in flight
static_assert(kPW % 4 == 0, "the reduced state's vector box moves four columns per innermost run");
constexpr int kRedVecPlanes = 3, kRedSclPlanes = 6;

// Pulled population of colour k, direction i, from the reduced state of its
// source node (phk = phi_k, fd = f^dagger_i, (vx, vy) = V_k there): Eq. 6 as
// the step's C stage forms it for the FP32 storage, the same FP32 operations
// in the same order, so the reduced state carries the FP32 form's
// populations bit for bit.  wrec: the recolouring weights w'_i.
__device__ __forceinline__ float red_pop(int i, float phk, float fd, float vx, float vy, const float* wrec) {
  switch (i) {
    case 0: return __fmul_rn(phk, fd);
    case 1: return __fmaf_rn(phk, fd, __fmul_rn(wrec[1], vx));
    case 2: return __fmaf_rn(phk, fd, __fmul_rn(wrec[2], vy));
    case 3: return __fmaf_rn(phk, fd, -__fmul_rn(wrec[1], vx));
    case 4: return __fmaf_rn(phk, fd, -__fmul_rn(wrec[2], vy));
    case 5: return __fmaf_rn(phk, fd, __fmul_rn(wrec[5], __fadd_rn(vx, vy)));
    case 6: return __fmaf_rn(phk, fd, __fmul_rn(wrec[6], __fsub_rn(vy, vx)));
    case 7: return __fmaf_rn(phk, fd, -__fmul_rn(wrec[5], __fadd_rn(vx, vy)));
    default: return __fmaf_rn(phk, fd, -__fmul_rn(wrec[6], __fsub_rn(vy, vx)));
  }
}
constexpr int kDW = kTX + 4;      // density/phi window:     x0-2 .. x0+w+2
constexpr int kTW = kTX + 2;      // tension-tensor window:  x0-1 .. x0+w+1
constexpr int kSlots = 4;         // population ring depth (rows): a row is free again after its D stage
constexpr int kMaxSlots = 6;      // barriers per ring (kSlots, or kRedSlots for the reduced state)
static_assert(kRedSlots <= kMaxSlots && kRedSlots * kRedSlotFloats <= kSlots * 3 * kGroupFloats,
              "the reduced ring must fit the FP32 ring");
constexpr int kConsumers = 256;   // 8 compute warps: one C-stage node each per pair of rows
constexpr int kThreads = kConsumers + 32;  // + 1 copy-issuing warp

// Strip s of n over nx columns: equal widths up to 4 columns, every edge on
// a multiple of 4 (n = ceil(nx / kTX) keeps every width <= kTX).  Used for
// batched instances, whose small grids would otherwise get sliver strips.
__host__ __device__ inline int strip_x0(int s, int n, int nx) { return 4 * ((s * (nx / 4)) / n); }

struct StepArgs {
  const float* fin;   // stored post-collision populations at t-1, [27][ny][P] (padded layout)
  float* fout;        // written at t (MODE_STEP), same layout
  int nx, ny;
  int pitch;          // P = pitch_of(nx)
  int boxw;           // FP32 TMA box width in columns (kPW)
  // 16-bit deviation storage: deviation planes [27][ny][P] and rho' planes
  // [3][ny][P] of the input and output buffers (unused for FP32)
  const unsigned short* din;
  unsigned short* dout;
  const float* rin;
  float* rout;
  int nstrips;        // ceil(nx / kTX)
  int rows_per_cta;   // H of the full-width strips
  int rows_last;      // H of the narrower last strip (when kTX does not divide nx)
  int full_blocks;    // CTAs of the full-width strips, (nx / kTX) * ceil(ny / H); the rest take the last strip
  float inv_nu[3];    // 1/nu_k, nu_k = (tau_k - 1/2)/3 (so 1/nu = sum_k phi_k/nu_k)
  float cpair[3];     // 1e6 / (rho0_k rho0_l) for pairs (12, 13, 23)
  float sigma[3];     // sigma_12, sigma_13, sigma_23
  float beta0;
  float beta_A;       // beta_kl = beta0 (1 + min(beta_A * r g b / rho^3, 1) * beta_h[kl])
  float beta_h[3];
  float wrec[9];      // recolouring weight per direction: w_i / |e_i|^p
  float ndelta;       // recolouring normal G / max(|G|, ndelta phi_k phi_l); 0 = G/|G|
  unsigned int* err;  // device error word (bit 0: a bounded wait timed out)
  int stall_row;      // testing hook: CTA 0's producer skips the copies of this march row (-1: none)
  // MODE_FIELDS outputs (FP64, [3][N] and [N]); NULL entries are skipped
  double* out_rho;
  double* out_ux;
  double* out_uy;
  double* out_p;
};

enum { MODE_STEP = 0, MODE_FIELDS = 1 };

// ------------------------------------------------------ batched launches
// One CTA tile of one instance.
struct BatchItem {
  int inst;
  int x0, w, y0, h;
};
// Per instance: step arguments and TMA descriptor for each buffer parity
// (parity p reads buffer p and writes buffer 1 - p).
// map[p] holds the input buffer's TMA descriptors (two for the reduced
// state: vector and scalar planes).  A reduced-state instance whose state is
// still FP32 populations (after it was set) steps once with args_f2r[p]
// (its FP32 populations in, the reduced state out) and map_f2r.
struct alignas(64) BatchDesc {
  StepArgs args[2];
  StepArgs args_f2r[2];
  alignas(64) unsigned char map[2][256];
  alignas(64) unsigned char map_f2r[256];
};
// The step arguments of up to kBatchParamInst instances for one parity,
// passed by value in the kernel parameter space (at most 32,764 bytes on
// sm_70 and later): each argument is then a read of the constant bank at an
// index uniform over the CTA, as for the single grid.  Larger batches read
// them from the BatchDesc array in global memory.
constexpr int kBatchParamInst = 144;
struct BatchArgsBlock {
  StepArgs a[kBatchParamInst];
};
static_assert(sizeof(BatchArgsBlock) + 64 <= 32764, "kernel parameter space");

size_t step_smem_bytes();
cudaError_t step_configure();  // sets the dynamic shared memory attribute
// tmaps: two CUtensorMaps (128 bytes each) of the input buffer: FP32 storage
// uses the first, a (P, ny, 27) FP32 tensor with box (kPW, 1, 9); 16-bit
// storage uses both, the (P, ny, 27) deviation tensor with box
// (kDevBoxCols, 1, 9) and the (P, ny, 3) FP32 rho' tensor with box (kPW, 1, 3).
// force: 0 = the force of Eq. 11 through Guo's term (Eq. 5); 1 = the
// perturbation operator of Eqs. phi1 / phi_old (FP32 storage only)
cudaError_t launch_step(const StepArgs& a, const void* tmaps, int grid, int mode, int storage, int force,
                        cudaStream_t s);
// encode those maps for one population buffer (uses the driver's encoder)
cudaError_t encode_population_maps(void* tmaps, const void* buf, int nx, int ny, int storage);
// bytes of one population buffer
size_t population_bytes(int nx, int ny, int storage);
// args: this parity's arguments of every instance (count <= kBatchParamInst),
// or nullptr to read them from descs
// storage: ST_FP32 or ST_RED for the steps of the batch; ST_F2R for the
// first step of reduced-state instances set from populations (descs' F2R
// arguments, read from global memory)
cudaError_t launch_batch(const BatchItem* items, int nitems, const BatchDesc* descs, const BatchArgsBlock* args,
                         int parity, int storage, cudaStream_t s);
int step_occupancy(int* blocks_per_sm);

// ------------------------------------------------------------- aux kernels
cudaError_t launch_init_from_rho(const double* rho, float* f, int nx, int ny, cudaStream_t s);
cudaError_t launch_set_planes(const double* fpost, float* f, int nx, int ny, int plane0, int nplanes,
                              cudaStream_t s);
cudaError_t launch_get_planes(const float* f, double* fpost, int nx, int ny, int plane0, int nplanes,
                              cudaStream_t s);
cudaError_t launch_check_rho(const double* rho, int n, unsigned int* bad, cudaStream_t s);
// 16-bit storage: FP32 padded stored values <-> deviations + rho'
cudaError_t launch_encode(const float* fp32, void* buf, int nx, int ny, int storage, cudaStream_t s);
cudaError_t launch_decode(const void* buf, float* fp32, int nx, int ny, int storage, cudaStream_t s);
// reduced state -> FP32 stored populations (padded layout); a.wrec are the recolouring weights
cudaError_t launch_expand_reduced(const float* red, float* fp32, int nx, int ny, const StepArgs& a,
                                  cudaStream_t s);
cudaError_t launch_reduce_dev(const void* buf, int nx, int ny, int storage, double* partial, int blocks,
                              double* out, cudaStream_t s);
// FP64 reductions: partial[blocks][5] then out[5] = (mass_r, mass_g, mass_b, mom_x, mom_y)
int reduce_blocks(int N);
// plain [27][ny][nx] array, plane = k*9 + i (the allocation-free entry point's input)
cudaError_t launch_reduce(const float* f, int N, double* partial, int blocks, double* out, cudaStream_t s);
// the library's padded, group-ordered layout
cudaError_t launch_reduce_padded(const float* f, int nx, int ny, double* partial, int blocks, double* out,
                                 cudaStream_t s);

// ------------------------------------------------ interface diagnostics
// FP64 interface points, circle moments and bulk pressure sums of FP64
// fields rho [3][N], p [N] (lbm3_diag.cu): partial sums of up to
// kDiagMaxBlocks blocks, then the 33 totals at scratch + kDiagMaxBlocks * 33.
constexpr int kDiagMaxBlocks = 1024;
size_t diag_scratch_doubles();
cudaError_t launch_diag(const double* rho, const double* p, int nx, int ny, double third_max, double bulk_min,
                        double* scratch, cudaStream_t s);
// host side: circles, junctions and contact angles from the 33 totals
using DiagResult = lbm3_interfaces;
void diag_geometry(const double* sums, int nx, int ny, DiagResult* r);

}  // namespace lbm3
