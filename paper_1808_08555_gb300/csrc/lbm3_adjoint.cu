// Reverse mode (adjoint) of the fused step: hand-written vector-Jacobian
// products of the ternary colour-gradient update (arXiv 1808.08555, Sec. 2),
// for gradients of a loss of the colour fractions with respect to the
// initial state and the interfacial tensions.
//
// One step maps the stored post-collision state S_{t-1} to S_t.  Its
// adjoint, given the cotangent L_t = dJ/dS_t, is taken as a chain of
// gathers, each node written by exactly one thread:
//   recompute:  rho_k (pulled densities), grad phi_k (Eq. fd1) and the
//               tension tensor T (Eq. 11) of S_{t-1};
//   node VJP:   collision with the Guo force and recolouring (Eqs. 1-3, 5,
//               6, uk1, vis_1, tau, 18-20) at each node -> cotangents of the
//               total distribution f_i, of rho_k, of grad phi_k and of F_s;
//   tension:    F_s = div T transposed (a gather), then T's dependence on
//               phi, grad phi, rho_k (through C_kl) and sigma;
//   gradient:   Eq. fd1 transposed: dJ/dphi_k(y) = sum_j c_j e_j . dJ/d(grad phi_k)(y - e_j);
//   pull:       L_{t-1,ik}(z) = dJ/df_ik(z + e_i), the transpose of streaming.
// The cotangent of the pulled populations is kept factored as
// dJ/df_ik(x) = lam9_i(x) + lamr_k(x) (total-distribution and density
// parts), so the pull of the next (earlier) step is folded into its node VJP,
// which reads lam9 and lamr at x + e_i: no 27-plane cotangent array exists.
// Three launches per step: node VJP; tension VJP beside the densities of the
// next state to differentiate; gradient VJP beside that state's grad phi and
// T (the recompute of step t-1 is independent of the cotangents of step t,
// so it rides in the same launches as extra blocks).
// All arithmetic is FP32 (the recomputed forward quantities and the
// cotangents); the scalar gradients are summed per block in FP32 and added
// in FP64 to a block-owned row, so the result does not depend on scheduling.
//
// Array conventions: per-node fields are [c][ny][nx] arrays; the tape states
// are in the library's padded, group-ordered layout.

#include <cmath>
#include <cstdint>

#include "lbm3_adjoint.h"
#include "lbm3_internal.h"

namespace lbm3 {
namespace {

constexpr int kAdjThreads = 256;

// Programmatic dependent launch: the adjoint's kernels are launched with
// programmatic stream serialisation, so a kernel's launch and prologue
// overlap the tail of the one before it.  Each waits here until its
// predecessor grid has completed and its writes are visible, then lets its
// own successor launch.  The wait always ends: the predecessor does not wait
// on this grid, and a successor starts only once every block of this grid is
// resident.
__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// periodic wrap of a coordinate at most one cell outside [0, n)
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ int nbr(int x, int y, int dx, int dy, int nx, int ny) {
  return wrap1(y + dy, ny) * nx + wrap1(x + dx, nx);
}

// pulled population f_{i,k}(x) = stored_{i,k}(x - e_i) of a padded state;
// the ghost columns hold the periodic copies, so only the row wraps
__device__ __forceinline__ float pulled(const float* __restrict__ st, int k, int i, int x, int y, int nx, int ny,
                                        size_t PS, int P) {
  (void)nx;
  return st[plane_of(k, i) * PS + static_cast<size_t>(wrap1(y - ey(i), ny)) * P + (x - ex(i) + kGhost)];
}

// Sum three values over the block and add the totals to row[0..2] in FP64
// (the row belongs to this block only).  The in-block tree is FP32 (8 levels,
// relative error ~5e-7 of the block total): FP64 arithmetic is a small
// fraction of the FP32 rate on this GPU, and an FP64 tree per thread would
// cost more than the kernel's memory traffic.  Every thread must call it.
__device__ __forceinline__ void block_add3(float v0, float v1, float v2, double* row) {
  __shared__ float sh[3][kAdjThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, off);
    v1 += __shfl_down_sync(0xffffffffu, v1, off);
    v2 += __shfl_down_sync(0xffffffffu, v2, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][warp] = v0;
    sh[1][warp] = v1;
    sh[2][warp] = v2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < kAdjThreads / 32; ++w) s += sh[threadIdx.x][w];
    row[threadIdx.x] += static_cast<double>(s);
  }
}

// ------------------------------------------------------------- recompute
__device__ __forceinline__ void density_node(const float* __restrict__ st, float* __restrict__ rho3, int n, int nx,
                                             int ny) {
  const int N = nx * ny;
  const int x = n % nx, y = n / nx, P = pitch_of(nx);
  const size_t PS = static_cast<size_t>(P) * ny;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) s += pulled(st, k, i, x, y, nx, ny, PS, P);
    rho3[static_cast<size_t>(k) * N + n] = s;
  }
}

// grad phi_k (Eq. fd1) and T = sum_pairs sigma C |G| (I - n n) (Eq. 11)
__device__ __forceinline__ void tension_fwd_node(const float* __restrict__ rho3, float* __restrict__ gphi,
                                                 float* __restrict__ T, const StepArgs& a, int n) {
  const int nx = a.nx, ny = a.ny, N = nx * ny;
  const int x = n % nx, y = n / nx;
  float gx[3] = {0.0f, 0.0f, 0.0f}, gy[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int j = 1; j < 9; ++j) {
    const int m = nbr(x, y, ex(j), ey(j), nx, ny);
    const float r0 = rho3[m], r1 = rho3[static_cast<size_t>(N) + m], r2 = rho3[2 * static_cast<size_t>(N) + m];
    const float ir = 1.0f / (r0 + r1 + r2);
    const float c = 3.0f * wt(j);
    const float ph[3] = {r0 * ir, r1 * ir, r2 * ir};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gx[k] += c * ex(j) * ph[k];
      gy[k] += c * ey(j) * ph[k];
    }
  }
  const float rk[3] = {rho3[n], rho3[static_cast<size_t>(N) + n], rho3[2 * static_cast<size_t>(N) + n]};
  const float ir = 1.0f / (rk[0] + rk[1] + rk[2]);
  const float ph[3] = {rk[0] * ir, rk[1] * ir, rk[2] * ir};
  float txx = 0.0f, txy = 0.0f, tyy = 0.0f;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int k = p < 2 ? 0 : 1, l = p == 0 ? 1 : 2;
    const float Gx = ph[l] * gx[k] - ph[k] * gx[l];
    const float Gy = ph[l] * gy[k] - ph[k] * gy[l];
    const float g2 = Gx * Gx + Gy * Gy;
    if (g2 > 1e-30f) {
      const float ck = fminf(a.cpair[p] * rk[k] * rk[l], 1.0f);
      const float sc = a.sigma[p] * ck / sqrtf(g2);
      txx += sc * Gy * Gy;
      txy -= sc * Gx * Gy;
      tyy += sc * Gx * Gx;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gphi[static_cast<size_t>(2 * k) * N + n] = gx[k];
    gphi[static_cast<size_t>(2 * k + 1) * N + n] = gy[k];
  }
  T[n] = txx;
  T[static_cast<size_t>(N) + n] = txy;
  T[2 * static_cast<size_t>(N) + n] = tyy;
}

__global__ void __launch_bounds__(kAdjThreads) adj_density_kernel(const float* __restrict__ st,
                                                                  float* __restrict__ rho3, int nx, int ny) {
  pdl_wait_then_release();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nx * ny) density_node(st, rho3, n, nx, ny);
}

__global__ void __launch_bounds__(kAdjThreads) adj_tension_fwd_kernel(const float* __restrict__ rho3,
                                                                      float* __restrict__ gphi,
                                                                      float* __restrict__ T, StepArgs a) {
  pdl_wait_then_release();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < a.nx * a.ny) tension_fwd_node(rho3, gphi, T, a, n);
}

// ------------------------------------------------------------- node VJP
// The cotangent of the step's output stored at x is that of the pulled
// populations of the later step at x + e_i: L_ik(x) = lam9p_i(x + e_i) +
// lamrp_k(x + e_i).  Writes the cotangents of the total distribution f_i
// (lam9), of rho_k (lamr, including every dependence through phi_k, rho and
// beta), of grad phi_k (lamg) and of F_s (lamF); adds sum dJ/dh_q (the
// per-pair beta coefficients) to acc[3..5].
__global__ void __launch_bounds__(kAdjThreads, 3) adj_node_kernel(const float* __restrict__ st,
                                                               const float* __restrict__ gphi,
                                                               const float* __restrict__ T,
                                                               const float* __restrict__ lam9p,
                                                               const float* __restrict__ lamrp,
                                                               float* __restrict__ lam9, float* __restrict__ lamr,
                                                               float* __restrict__ lamg, float* __restrict__ lamF,
                                                               double* __restrict__ acc, StepArgs a) {
  pdl_wait_then_release();
  const int nx = a.nx, ny = a.ny, N = nx * ny;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  float dh0 = 0.0f, dh1 = 0.0f, dh2 = 0.0f;
  if (n < N) {
    const int x = n % nx, y = n / nx, P = pitch_of(nx);
    const size_t PS = static_cast<size_t>(P) * ny;
    // ---- forward recompute at this node
    float fi[9], rk[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float f0 = pulled(st, 0, i, x, y, nx, ny, PS, P);
      const float f1 = pulled(st, 1, i, x, y, nx, ny, PS, P);
      const float f2 = pulled(st, 2, i, x, y, nx, ny, PS, P);
      rk[0] += f0;
      rk[1] += f1;
      rk[2] += f2;
      fi[i] = f0 + f1 + f2;
    }
    const float rho = rk[0] + rk[1] + rk[2];
    const float ir = 1.0f / rho;
    const float ph[3] = {rk[0] * ir, rk[1] * ir, rk[2] * ir};
    float Fx = 0.0f, Fy = 0.0f;
#pragma unroll
    for (int j = 1; j < 9; ++j) {
      const int m = nbr(x, y, ex(j), ey(j), nx, ny);
      const float c = 3.0f * wt(j);
      Fx += c * (ex(j) * T[m] + ey(j) * T[static_cast<size_t>(N) + m]);
      Fy += c * (ex(j) * T[static_cast<size_t>(N) + m] + ey(j) * T[2 * static_cast<size_t>(N) + m]);
    }
    float mx = 0.0f, my = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      mx += ex(i) * fi[i];
      my += ey(i) * fi[i];
    }
    const float ux = (mx + 0.5f * Fx) * ir, uy = (my + 0.5f * Fy) * ir;
    const float inu = ph[0] * a.inv_nu[0] + ph[1] * a.inv_nu[1] + ph[2] * a.inv_nu[2];
    const float dom = 3.0f + 0.5f * inu;
    const float om = inu / dom;  // 1/tau_f
    const float g = 1.0f - 0.5f * om;
    const float uu = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
    float feq[9], Ai[9], fd[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float eu = ex(i) * ux + ey(i) * uy, eF = ex(i) * Fx + ey(i) * Fy;
      feq[i] = wt(i) * rho * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
      Ai[i] = 3.0f * eF - 3.0f * uF + 9.0f * eu * eF;  // Guo: Phi_i = w_i g A_i
      fd[i] = fi[i] + om * (feq[i] - fi[i]) + g * wt(i) * Ai[i];
    }
    const float prod = ph[0] * ph[1] * ph[2];
    const float cbr = a.beta_A * prod, cb = fminf(cbr, 1.0f);
    float gpx[3], gpy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gpx[k] = gphi[static_cast<size_t>(2 * k) * N + n];
      gpy[k] = gphi[static_cast<size_t>(2 * k + 1) * N + n];
    }
    // ---- reverse: recolouring (Eq. 6)
    float lfd[9], lph[3] = {0.0f, 0.0f, 0.0f}, mux[3] = {0.0f, 0.0f, 0.0f}, muy[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int m = nbr(x, y, ex(i), ey(i), nx, ny);
      const float l9 = lam9p[static_cast<size_t>(i) * N + m];
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float L = l9 + lamrp[static_cast<size_t>(k) * N + m];
        s += ph[k] * L;
        lph[k] += fd[i] * L;
        mux[k] += a.wrec[i] * ex(i) * L;
        muy[k] += a.wrec[i] * ey(i) * L;
      }
      lfd[i] = s;
    }
    float lrho = 0.0f, lcb = 0.0f;
    float lgx[3] = {0.0f, 0.0f, 0.0f}, lgy[3] = {0.0f, 0.0f, 0.0f};
    float dh[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const int k = p < 2 ? 0 : 1, l = p == 0 ? 1 : 2;
      const float Gx = ph[l] * gpx[k] - ph[k] * gpx[l];
      const float Gy = ph[l] * gpy[k] - ph[k] * gpy[l];
      const float g2 = Gx * Gx + Gy * Gy;
      if (!(g2 > 1e-30f)) continue;  // no k-l interface: n = 0
      const float mag = sqrtf(g2);
      const float pp = ph[k] * ph[l];
      const float den = fmaxf(mag, a.ndelta * pp);  // recolouring normal G / max(|G|, delta phi_k phi_l)
      const float nxv = Gx / den, nyv = Gy / den;
      const float b = a.beta0 * (1.0f + cb * a.beta_h[p]);
      const float amp = b * pp * rho;  // beta_kl rho_k rho_l / rho
      // colour k gains amp n . e_i w'_i, colour l loses it
      const float vx = mux[k] - mux[l], vy = muy[k] - muy[l];
      const float lamp = nxv * vx + nyv * vy;
      const float lnx = amp * vx, lny = amp * vy;
      const float lb = lamp * pp * rho;
      lph[k] += lamp * b * ph[l] * rho;
      lph[l] += lamp * b * ph[k] * rho;
      lrho += lamp * b * pp;
      lcb += lb * a.beta0 * a.beta_h[p];
      dh[p] = lb * a.beta0 * cb;
      float lGx, lGy;
      if (mag >= a.ndelta * pp) {  // unit normal G/|G|
        const float nl = nxv * lnx + nyv * lny;
        lGx = (lnx - nxv * nl) / mag;
        lGy = (lny - nyv * nl) / mag;
      } else {  // G / (delta phi_k phi_l)
        lGx = lnx / den;
        lGy = lny / den;
        const float lden = -(lnx * nxv + lny * nyv) / den;
        lph[k] += lden * a.ndelta * ph[l];
        lph[l] += lden * a.ndelta * ph[k];
      }
      // G = phi_l grad phi_k - phi_k grad phi_l
      lgx[k] += ph[l] * lGx;
      lgy[k] += ph[l] * lGy;
      lgx[l] -= ph[k] * lGx;
      lgy[l] -= ph[k] * lGy;
      lph[l] += gpx[k] * lGx + gpy[k] * lGy;
      lph[k] -= gpx[l] * lGx + gpy[l] * lGy;
    }
    dh0 = dh[0];
    dh1 = dh[1];
    dh2 = dh[2];
    if (cbr < 1.0f) {  // c = min(A phi_1 phi_2 phi_3, 1) (Eq. 19)
      lph[0] += lcb * a.beta_A * ph[1] * ph[2];
      lph[1] += lcb * a.beta_A * ph[0] * ph[2];
      lph[2] += lcb * a.beta_A * ph[0] * ph[1];
    }
    // ---- reverse: BGK collision with the Guo force
    float lfi[9], lom = 0.0f, lux = 0.0f, luy = 0.0f, lFx = 0.0f, lFy = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      lfi[i] = (1.0f - om) * lfd[i];
      lom += lfd[i] * (feq[i] - fi[i] - 0.5f * wt(i) * Ai[i]);
      const float lfeq = om * lfd[i], lA = g * wt(i) * lfd[i];
      const float eu = ex(i) * ux + ey(i) * uy, eF = ex(i) * Fx + ey(i) * Fy;
      lFx += lA * (3.0f * ex(i) - 3.0f * ux + 9.0f * eu * ex(i));
      lFy += lA * (3.0f * ey(i) - 3.0f * uy + 9.0f * eu * ey(i));
      lux += lA * (-3.0f * Fx + 9.0f * eF * ex(i));
      luy += lA * (-3.0f * Fy + 9.0f * eF * ey(i));
      lrho += lfeq * feq[i] * ir;
      const float wr = wt(i) * rho * lfeq;
      lux += wr * (3.0f * ex(i) + 9.0f * eu * ex(i) - 3.0f * ux);
      luy += wr * (3.0f * ey(i) + 9.0f * eu * ey(i) - 3.0f * uy);
    }
    // omega = inu / (3 + inu/2), inu = sum_k phi_k / nu_k (Eqs. vis_1, tau)
    const float linu = lom * 3.0f / (dom * dom);
#pragma unroll
    for (int k = 0; k < 3; ++k) lph[k] += linu * a.inv_nu[k];
    // u = (m + F/2) / rho (Eq. uk1)
    const float lmx = lux * ir, lmy = luy * ir;
    lFx += 0.5f * lmx;
    lFy += 0.5f * lmy;
    lrho -= (lux * ux + luy * uy) * ir;
#pragma unroll
    for (int i = 1; i < 9; ++i) lfi[i] += lmx * ex(i) + lmy * ey(i);
    // phi_k = rho_k / rho, rho = sum_k rho_k
    const float sph = ph[0] * lph[0] + ph[1] * lph[1] + ph[2] * lph[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) lamr[static_cast<size_t>(k) * N + n] = (lph[k] - sph) * ir + lrho;
#pragma unroll
    for (int i = 0; i < 9; ++i) lam9[static_cast<size_t>(i) * N + n] = lfi[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lamg[static_cast<size_t>(2 * k) * N + n] = lgx[k];
      lamg[static_cast<size_t>(2 * k + 1) * N + n] = lgy[k];
    }
    lamF[n] = lFx;
    lamF[static_cast<size_t>(N) + n] = lFy;
  }
  block_add3(dh0, dh1, dh2, acc + static_cast<size_t>(blockIdx.x) * 6 + 3);
}

// ------------------------------------------------------------ tension VJP
// dJ/dT from dJ/dF_s (the divergence of Eq. 11 transposed), then T's
// dependence on grad phi_k, phi_k, rho_k (C_kl) and sigma_kl.  Adds to
// lamg and lamr of this node; ds_out = this node's dJ/dsigma_q.
__device__ __forceinline__ void tension_vjp_node(const float* __restrict__ rho3, const float* __restrict__ gphi,
                                                 const float* __restrict__ lamF, float* __restrict__ lamg,
                                                 float* __restrict__ lamr, const StepArgs& a, int n,
                                                 float* ds_out) {
  const int nx = a.nx, ny = a.ny, N = nx * ny;
  const int x = n % nx, y = n / nx;
  float lxx = 0.0f, lxy = 0.0f, lyy = 0.0f;
#pragma unroll
  for (int j = 1; j < 9; ++j) {
    const int m = nbr(x, y, -ex(j), -ey(j), nx, ny);
    const float c = 3.0f * wt(j), Lx = lamF[m], Ly = lamF[static_cast<size_t>(N) + m];
    lxx += c * ex(j) * Lx;
    lxy += c * (ey(j) * Lx + ex(j) * Ly);
    lyy += c * ey(j) * Ly;
  }
  const float rk[3] = {rho3[n], rho3[static_cast<size_t>(N) + n], rho3[2 * static_cast<size_t>(N) + n]};
  const float ir = 1.0f / (rk[0] + rk[1] + rk[2]);
  const float ph[3] = {rk[0] * ir, rk[1] * ir, rk[2] * ir};
  float gpx[3], gpy[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gpx[k] = gphi[static_cast<size_t>(2 * k) * N + n];
    gpy[k] = gphi[static_cast<size_t>(2 * k + 1) * N + n];
  }
  float lph[3] = {0.0f, 0.0f, 0.0f}, lrk[3] = {0.0f, 0.0f, 0.0f};
  float lgx[3] = {0.0f, 0.0f, 0.0f}, lgy[3] = {0.0f, 0.0f, 0.0f};
  float ds[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int k = p < 2 ? 0 : 1, l = p == 0 ? 1 : 2;
    const float Gx = ph[l] * gpx[k] - ph[k] * gpx[l];
    const float Gy = ph[l] * gpy[k] - ph[k] * gpy[l];
    const float g2 = Gx * Gx + Gy * Gy;
    if (!(g2 > 1e-30f)) continue;
    // with m = |G| and the unit normal n = G/m: T_q = sigma C m (ny^2, -nx ny, nx^2),
    // dJ/dT : T_q = sigma C m q with q = lxx ny^2 - lxy nx ny + lyy nx^2, and
    // d(m q)/dG = (2 lyy nx - lxy ny - q nx, 2 lxx ny - lxy nx - q ny): no
    // negative powers of m, which would overflow FP32 where |G| is tiny
    const float m = sqrtf(g2), nxv = Gx / m, nyv = Gy / m;
    const float cr = a.cpair[p] * rk[k] * rk[l], ck = fminf(cr, 1.0f);
    const float q = lxx * nyv * nyv - lxy * nxv * nyv + lyy * nxv * nxv;
    ds[p] = ck * m * q;
    const float lck = a.sigma[p] * m * q;
    if (cr < 1.0f) {
      lrk[k] += lck * a.cpair[p] * rk[l];
      lrk[l] += lck * a.cpair[p] * rk[k];
    }
    const float aa = a.sigma[p] * ck;
    const float lGx = aa * (2.0f * lyy * nxv - lxy * nyv - q * nxv);
    const float lGy = aa * (2.0f * lxx * nyv - lxy * nxv - q * nyv);
    lgx[k] += ph[l] * lGx;
    lgy[k] += ph[l] * lGy;
    lgx[l] -= ph[k] * lGx;
    lgy[l] -= ph[k] * lGy;
    lph[l] += gpx[k] * lGx + gpy[k] * lGy;
    lph[k] -= gpx[l] * lGx + gpy[l] * lGy;
  }
  ds_out[0] = ds[0];
  ds_out[1] = ds[1];
  ds_out[2] = ds[2];
  const float sph = ph[0] * lph[0] + ph[1] * lph[1] + ph[2] * lph[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lamr[static_cast<size_t>(k) * N + n] += (lph[k] - sph) * ir + lrk[k];
    lamg[static_cast<size_t>(2 * k) * N + n] += lgx[k];
    lamg[static_cast<size_t>(2 * k + 1) * N + n] += lgy[k];
  }
}

// --------------------------------------------------- gradient stencil VJP
__device__ __forceinline__ void grad_vjp_node(const float* __restrict__ rho3, const float* __restrict__ lamg,
                                              float* __restrict__ lamr, int nx, int ny, int n) {
  const int N = nx * ny;
  const int x = n % nx, y = n / nx;
  float lph[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int j = 1; j < 9; ++j) {
    const int m = nbr(x, y, -ex(j), -ey(j), nx, ny);
    const float c = 3.0f * wt(j);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      lph[k] += c * (ex(j) * lamg[static_cast<size_t>(2 * k) * N + m] +
                     ey(j) * lamg[static_cast<size_t>(2 * k + 1) * N + m]);
  }
  const float rk[3] = {rho3[n], rho3[static_cast<size_t>(N) + n], rho3[2 * static_cast<size_t>(N) + n]};
  const float ir = 1.0f / (rk[0] + rk[1] + rk[2]);
  const float sph = (rk[0] * lph[0] + rk[1] * lph[1] + rk[2] * lph[2]) * ir;
#pragma unroll
  for (int k = 0; k < 3; ++k) lamr[static_cast<size_t>(k) * N + n] += (lph[k] - sph) * ir;
}

// Blocks [0, G): tension VJP of this step (acc row = block).  Blocks [G, 2G)
// when st_next is set: densities of the next state to differentiate.
__global__ void __launch_bounds__(kAdjThreads) adj_tension_kernel(const float* __restrict__ rho3,
                                                                  const float* __restrict__ gphi,
                                                                  const float* __restrict__ lamF,
                                                                  float* __restrict__ lamg, float* __restrict__ lamr,
                                                                  double* __restrict__ acc, StepArgs a, int G,
                                                                  const float* __restrict__ st_next,
                                                                  float* __restrict__ rho3_next) {
  pdl_wait_then_release();
  const int N = a.nx * a.ny;
  if (static_cast<int>(blockIdx.x) < G) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    float ds[3] = {0.0f, 0.0f, 0.0f};
    if (n < N) tension_vjp_node(rho3, gphi, lamF, lamg, lamr, a, n, ds);
    block_add3(ds[0], ds[1], ds[2], acc + static_cast<size_t>(blockIdx.x) * 6);
  } else {
    const int n = (blockIdx.x - G) * blockDim.x + threadIdx.x;
    if (n < N) density_node(st_next, rho3_next, n, a.nx, a.ny);
  }
}

// Blocks [0, G): gradient-stencil VJP of this step.  Blocks [G, 2G) when
// the next state's densities exist: its grad phi and T.
__global__ void __launch_bounds__(kAdjThreads) adj_grad_kernel(const float* __restrict__ rho3,
                                                               const float* __restrict__ lamg,
                                                               float* __restrict__ lamr, StepArgs a, int G,
                                                               const float* __restrict__ rho3_next,
                                                               float* __restrict__ gphi_next,
                                                               float* __restrict__ T_next) {
  pdl_wait_then_release();
  const int N = a.nx * a.ny;
  if (static_cast<int>(blockIdx.x) < G) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) grad_vjp_node(rho3, lamg, lamr, a.nx, a.ny, n);
  } else {
    const int n = (blockIdx.x - G) * blockDim.x + threadIdx.x;
    if (n < N) tension_fwd_node(rho3_next, gphi_next, T_next, a, n);
  }
}

// -------------------------------------------------- loss-side and outputs
// phi_k of a stored state, FP64 (the colour fractions at the time the state
// is pulled into)
__global__ void phi_kernel(const float* __restrict__ st, double* __restrict__ phi, int nx, int ny) {
  const int N = nx * ny;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = n % nx, y = n / nx, P = pitch_of(nx);
  const size_t PS = static_cast<size_t>(P) * ny;
  float r[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) s += pulled(st, k, i, x, y, nx, ny, PS, P);
    r[k] = s;
  }
  const double rho = static_cast<double>(r[0]) + r[1] + r[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) phi[static_cast<size_t>(k) * N + n] = r[k] / rho;
}

// Cotangent of the pulled populations at the end of the run from dJ/dphi_k:
// lamr_k = dJ/drho_k = (dphi_k - sum_m phi_m dphi_m) / rho, lam9 = 0.
__global__ void adj_seed_kernel(const float* __restrict__ rho3, const double* __restrict__ dphi,
                                float* __restrict__ lamr, float* __restrict__ lam9, int N) {
  pdl_wait_then_release();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double r[3] = {rho3[n], rho3[static_cast<size_t>(N) + n], rho3[2 * static_cast<size_t>(N) + n]};
  const double ir = 1.0 / (r[0] + r[1] + r[2]);
  const double d[3] = {dphi[n], dphi[static_cast<size_t>(N) + n], dphi[2 * static_cast<size_t>(N) + n]};
  const double s = (r[0] * d[0] + r[1] * d[1] + r[2] * d[2]) * ir;
#pragma unroll
  for (int k = 0; k < 3; ++k) lamr[static_cast<size_t>(k) * N + n] = static_cast<float>((d[k] - s) * ir);
#pragma unroll
  for (int i = 0; i < 9; ++i) lam9[static_cast<size_t>(i) * N + n] = 0.0f;
}

// dJ/df_ik(x) = lam9_i(x) + lamr_k(x) of the post-streaming populations at
// t = 0, planes plane0 .. plane0 + gridDim.y - 1 (numbering k*9 + i) into out
__global__ void adj_dpop_kernel(const float* __restrict__ lam9, const float* __restrict__ lamr,
                                double* __restrict__ out, int N, int plane0) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int pl = plane0 + blockIdx.y, k = pl / 9, i = pl % 9;
  out[static_cast<size_t>(blockIdx.y) * N + n] =
      static_cast<double>(lam9[static_cast<size_t>(i) * N + n]) + lamr[static_cast<size_t>(k) * N + n];
}

// dJ/drho_k(x) for the rest equilibrium f_ik = w_i rho_k: sum_i w_i dJ/df_ik
__global__ void adj_drho_kernel(const float* __restrict__ lam9, const float* __restrict__ lamr,
                                double* __restrict__ out, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double w[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
  double s9 = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s9 += w[i == 0 ? 0 : (i < 5 ? 1 : 2)] * lam9[static_cast<size_t>(i) * N + n];
#pragma unroll
  for (int k = 0; k < 3; ++k) out[static_cast<size_t>(k) * N + n] = s9 + lamr[static_cast<size_t>(k) * N + n];
}

int blocks_for(int N) { return (N + kAdjThreads - 1) / kAdjThreads; }

template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), int grid, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kAdjThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<K>(args)...);
}

}  // namespace

int adj_blocks(int N) { return blocks_for(N); }

size_t adj_scratch_floats(int N) { return static_cast<size_t>(56) * N; }

void adj_layout(float* base, int N, AdjBuffers* b) {
  const size_t n = static_cast<size_t>(N);
  b->lam9[0] = base;
  b->lam9[1] = base + 9 * n;
  b->lamr[0] = base + 18 * n;
  b->lamr[1] = base + 21 * n;
  b->lamg = base + 24 * n;
  b->lamF = base + 30 * n;
  b->rho3[0] = base + 32 * n;
  b->rho3[1] = base + 35 * n;
  b->gphi[0] = base + 38 * n;
  b->gphi[1] = base + 44 * n;
  b->T[0] = base + 50 * n;
  b->T[1] = base + 53 * n;
}

cudaError_t launch_phi(const float* st, double* phi, int nx, int ny, cudaStream_t s) {
  phi_kernel<<<blocks_for(nx * ny), kAdjThreads, 0, s>>>(st, phi, nx, ny);
  return cudaGetLastError();
}

cudaError_t launch_adj_seed(const float* st_final, const double* dphi, const AdjBuffers& b, int lam, int nx, int ny,
                            cudaStream_t s) {
  const int N = nx * ny, g = blocks_for(N);
  float* scratch = b.rho3[1];
  cudaError_t e = launch_pdl(adj_density_kernel, g, s, st_final, scratch, nx, ny);
  if (e == cudaSuccess) e = launch_pdl(adj_seed_kernel, g, s, scratch, dphi, b.lamr[lam], b.lam9[lam], N);
  return e;
}

cudaError_t launch_adj_fields(const float* st, const StepArgs& a, const AdjBuffers& b, int slot, cudaStream_t s) {
  const int g = blocks_for(a.nx * a.ny);
  cudaError_t e = launch_pdl(adj_density_kernel, g, s, st, b.rho3[slot], a.nx, a.ny);
  if (e == cudaSuccess) e = launch_pdl(adj_tension_fwd_kernel, g, s, b.rho3[slot], b.gphi[slot], b.T[slot], a);
  return e;
}

cudaError_t launch_adj_step(const float* st_prev, const float* st_next, const StepArgs& a, const AdjBuffers& b,
                            int slot, int lam, double* acc, cudaStream_t s) {
  const int N = a.nx * a.ny, G = blocks_for(N);
  const int o = lam ^ 1, nslot = slot ^ 1;
  const int g2 = st_next ? 2 * G : G;
  cudaError_t e = launch_pdl(adj_node_kernel, G, s, st_prev, b.gphi[slot], b.T[slot], b.lam9[lam], b.lamr[lam],
                             b.lam9[o], b.lamr[o], b.lamg, b.lamF, acc, a);
  if (e == cudaSuccess)
    e = launch_pdl(adj_tension_kernel, g2, s, b.rho3[slot], b.gphi[slot], b.lamF, b.lamg, b.lamr[o], acc, a, G, st_next,
                   b.rho3[nslot]);
  if (e == cudaSuccess)
    e = launch_pdl(adj_grad_kernel, g2, s, b.rho3[slot], b.lamg, b.lamr[o], a, G, b.rho3[nslot], b.gphi[nslot],
                   b.T[nslot]);
  return e;
}

cudaError_t launch_adj_dpop(const AdjBuffers& b, int lam, double* out, int nx, int ny, int plane0, int nplanes,
                            cudaStream_t s) {
  const int N = nx * ny;
  adj_dpop_kernel<<<dim3(blocks_for(N), nplanes), kAdjThreads, 0, s>>>(b.lam9[lam], b.lamr[lam], out, N, plane0);
  return cudaGetLastError();
}

cudaError_t launch_adj_drho(const AdjBuffers& b, int lam, double* out, int nx, int ny, cudaStream_t s) {
  const int N = nx * ny;
  adj_drho_kernel<<<blocks_for(N), kAdjThreads, 0, s>>>(b.lam9[lam], b.lamr[lam], out, N);
  return cudaGetLastError();
}

}  // namespace lbm3
