// N-fluid colour-gradient step on D2Q9 (arXiv 1808.08555: Eq. 11 and the
// recolouring of Eq. 6 are written for any number of fluids; the paper
// simulates three).  A first CUDA path for 2 <= N <= kMaxFluids, as three
// kernels per step over global-memory intermediates, one node per thread:
//   densities:  pull the 9N populations (Eq. 30), rho_k, rho, phi_k (the
//               largest fraction as the complement of the others, so they
//               sum to 1 exactly), the total distribution f_i
//   tension:    grad phi_k (Eq. fd1), G_kl and C_kl (Eq. 15) for the
//               N(N-1)/2 pairs, the tension tensor of Eq. 11 summed over the
//               pairs, the recolouring normals n_kl = G / max(|G|, delta phi_k phi_l),
//               beta_kl and the recolouring vectors V_k = sum_{l != k} beta_kl
//               (rho_k rho_l / rho) n_kl (2N values instead of N(N-1) normal
//               components)
//   collide:    F_s = div T (Eq. fd1), u (Eq. uk1), tau_f (Eqs. vis_1, tau),
//               BGK with Guo's forcing (Eqs. 1-3, 5), recolouring (Eq. 6);
//               f^ddagger stored at the node that produced it
// beta_kl for N fluids (the paper gives Eqs. 18-20 for three):
//   beta_kl = beta^0 [1 + sum_{m != k,l} min(35 rho_k rho_l rho_m / rho^3, 1) g(X_kl^m)],
// with g(X_kl^m) of Eqs. 18 and 20 precomputed on the host; it is Eq. 19
// exactly for N = 3.  The fluid count is a template parameter, so every
// per-node array stays in registers.
//
// Layout: populations [N][9][ny][nx] FP32, unpadded, periodic by index
// arithmetic, or the reduced state below; intermediates: the tension tensor
// as one float4 (xx, xy, yy, 0) per node, the fractions phi as vector planes
// (kCK planes [ny][nx] of kCW floats, as a component of the reduced state),
// rho [ny][nx], f_i [9][ny][nx], V [2][N][ny][nx] (x components, then y).

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm3.h"
#include "lbm3_internal.h"

namespace lbm3 {
namespace {

constexpr int kMaxFluids = 6;
constexpr int kMaxPairs = kMaxFluids * (kMaxFluids - 1) / 2;
constexpr int kNThreads = 128;

struct NArgs {
  int nx, ny;
  float inv_nu[kMaxFluids];                   // 1/nu_k
  float sigma[kMaxPairs];                     // sigma_kl for pairs k < l in row order
  float cpair[kMaxPairs];                     // 1e6 / (rho0_k rho0_l)
  float gjunc[kMaxPairs][kMaxFluids];         // g(X_kl^m) (0 for m = k, l)
  float beta0, beta_A;                        // beta_A = 35 (0: Eq. fu, constant beta)
  float wrec[9];                              // recolouring weights w_i / |e_i|^p
  float ndelta;
};

__host__ __device__ constexpr int pair_index(int k, int l, int n) {  // k < l
  return k * n - k * (k + 1) / 2 + (l - k - 1);
}

__device__ __forceinline__ int wrapn(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Programmatic dependent launch: the step's kernels are launched with
// programmatic stream serialisation, so a kernel's launch overlaps the tail of
// the one before it.  Each waits here until its predecessor grid has completed
// and its writes are visible, then lets its own successor launch.  The wait
// always ends: the predecessor does not wait on this grid, and a successor
// starts only once every block of this grid is resident.
__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<K>(args)...);
}

// ---------------------------------------------------------- reduced state
// Collision (Eqs. 1-3, 5) uses only the total distribution and the colour
// densities, and the recolouring of Eq. 6 writes
//   f^ddagger_{i,k} = phi_k f^dagger_i + w'_i e_i . V_k,
//   V_k = sum_{l != k} beta_kl (rho_k rho_l / rho) n_kl,
// so a node's 9 N outputs are fixed by phi_k, V_k and f^dagger_i: 3 N + 9
// values.  Layout inside a population buffer, by component: the fractions
// phi_1..N, then the x components V_1x..V_Nx, then the y components, each as
// kCK vector planes [ny][nx] of kCW floats (float2 for N = 2, float4 above,
// unused slots zero), then 9 float planes f^dagger_i.  A pull from direction
// i loads the fractions and only the components e_i has.  All N vectors V_k
// are kept although they sum to zero, so that every population is rebuilt
// from exactly the values the collision used.
template <int N>
constexpr int kCW = N <= 2 ? 2 : 4;  // floats per stored vector
template <int N>
constexpr int kCK = (N + kCW<N> - 1) / kCW<N>;  // vectors per component
template <int N>
constexpr size_t kRedVec = static_cast<size_t>(3) * kCK<N> * kCW<N>;  // floats per node before the f^dagger planes

template <int N>
__device__ __forceinline__ void comp_store(float* __restrict__ g, size_t NN, size_t n, int c, const float (&v)[N]) {
#pragma unroll
  for (int j = 0; j < kCK<N>; ++j) {
    const size_t m = (static_cast<size_t>(c) * kCK<N> + j) * NN + n;
    float e[kCW<N>];
#pragma unroll
    for (int q = 0; q < kCW<N>; ++q) e[q] = kCW<N> * j + q < N ? v[(kCW<N> * j + q) % N] : 0.0f;
    if constexpr (kCW<N> == 2)
      reinterpret_cast<float2*>(g)[m] = make_float2(e[0], e[1]);
    else
      reinterpret_cast<float4*>(g)[m] = make_float4(e[0], e[1], e[2], e[3]);
  }
}

template <int N>
__device__ __forceinline__ void comp_load(const float* __restrict__ g, size_t NN, size_t n, int c, float (&v)[N]) {
#pragma unroll
  for (int j = 0; j < kCK<N>; ++j) {
    const size_t m = (static_cast<size_t>(c) * kCK<N> + j) * NN + n;
    float e[4];
    if constexpr (kCW<N> == 2) {
      const float2 w = reinterpret_cast<const float2*>(g)[m];
      e[0] = w.x;
      e[1] = w.y;
    } else {
      const float4 w = reinterpret_cast<const float4*>(g)[m];
      e[0] = w.x;
      e[1] = w.y;
      e[2] = w.z;
      e[3] = w.w;
    }
#pragma unroll
    for (int q = 0; q < kCW<N>; ++q)
      if (kCW<N> * j + q < N) v[(kCW<N> * j + q) % N] = e[q];
  }
}

// e_i . V over the nonzero components of e_i
__device__ __forceinline__ float edot2(int i, float vx, float vy) {
  const float a = ex(i) > 0 ? vx : -vx;
  const float b = ey(i) > 0 ? vy : -vy;
  if (ex(i) != 0) return ey(i) != 0 ? __fadd_rn(a, b) : a;
  return ey(i) != 0 ? b : 0.0f;
}

// Eq. 6 for one population, f^ddagger = phi_k f^dagger_i + w'_i (e_i . V_k),
// in explicitly rounded operations: the collision's store and the reduced
// state's rebuild give the same bits
__device__ __forceinline__ float recolour2(float phk, float fdi, float wr, float ev) {
  return __fmaf_rn(wr, ev, __fmul_rn(phk, fdi));
}

template <int N, bool RED>
__global__ void __launch_bounds__(kNThreads) n_density_kernel(const float* __restrict__ f, float* __restrict__ phi,
                                                              float* __restrict__ rho_out, float* __restrict__ fi,
                                                              NArgs a) {
  pdl_wait_then_release();
  const int nx = a.nx, ny = a.ny;
  const size_t NN = static_cast<size_t>(nx) * ny;
  {
    // one row per block row of the grid: no division for the node's coordinates
    const int y = static_cast<int>(blockIdx.x);
    const int x = static_cast<int>(blockIdx.y) * kNThreads + static_cast<int>(threadIdx.x);
    if (x >= nx) return;
    const size_t n = static_cast<size_t>(y) * nx + x;
    float r[N];
    float tot[9];
    if constexpr (RED) {
      // each pulled population rebuilt from its source node, then the sums of
      // the population form in the same order (the same bits)
      const float* __restrict__ fd = f + kRedVec<N> * NN;
      float fdv[9];
#pragma unroll
      for (int i = 0; i < 9; ++i)
        fdv[i] = fd[static_cast<size_t>(i) * NN + static_cast<size_t>(wrapn(y - ey(i), ny)) * nx + wrapn(x - ex(i), nx)];
#pragma unroll
      for (int k = 0; k < N; ++k) r[k] = 0.0f;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const size_t src = static_cast<size_t>(wrapn(y - ey(i), ny)) * nx + wrapn(x - ex(i), nx);
        float sp[N], svx[N], svy[N];
#pragma unroll
        for (int k = 0; k < N; ++k) svx[k] = svy[k] = 0.0f;
        comp_load<N>(f, NN, src, 0, sp);
        if (ex(i) != 0) comp_load<N>(f, NN, src, 1, svx);
        if (ey(i) != 0) comp_load<N>(f, NN, src, 2, svy);
        float t = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const float v = recolour2(sp[k], fdv[i], a.wrec[i], edot2(i, svx[k], svy[k]));
          r[k] += v;
          t += v;
        }
        tot[i] = t;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) tot[i] = 0.0f;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        // a colour's 9 pulled values (Eq. 30) loaded together, then summed
        float v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i)
          v[i] = f[(static_cast<size_t>(k) * 9 + i) * NN + static_cast<size_t>(wrapn(y - ey(i), ny)) * nx +
                   wrapn(x - ex(i), nx)];
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          s += v[i];
          tot[i] += v[i];
        }
        r[k] = s;
      }
    }
    float rho = 0.0f, rmax = -1.0f;
    int kmax = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      rho += r[k];
      if (r[k] > rmax) {
        rmax = r[k];
        kmax = k;
      }
    }
    const float ir = 1.0f / rho;
    float rest = 1.0f, ph[N];
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k != kmax) {
        ph[k] = r[k] * ir;
        rest -= ph[k];
      }
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k == kmax) ph[k] = rest;  // the fractions sum to 1 exactly
    comp_store<N>(phi, NN, n, 0, ph);
    rho_out[n] = rho;
#pragma unroll
    for (int i = 0; i < 9; ++i) fi[static_cast<size_t>(i) * NN + n] = tot[i];
  }
}

template <int N>
__global__ void __launch_bounds__(kNThreads) n_tension_kernel(const float* __restrict__ phi,
                                                              const float* __restrict__ rho_in, float4* __restrict__ T,
                                                              float* __restrict__ Vout, NArgs a) {
  pdl_wait_then_release();
  const int nx = a.nx, ny = a.ny;
  const size_t NN = static_cast<size_t>(nx) * ny;
  {
    // one row per block row of the grid: no division for the node's coordinates
    const int y = static_cast<int>(blockIdx.x);
    const int x = static_cast<int>(blockIdx.y) * kNThreads + static_cast<int>(threadIdx.x);
    if (x >= nx) return;
    const size_t n = static_cast<size_t>(y) * nx + x;
    float ph[N], gx[N], gy[N];
    comp_load<N>(phi, NN, n, 0, ph);
#pragma unroll
    for (int k = 0; k < N; ++k) gx[k] = gy[k] = 0.0f;
    // Eq. fd1: (1/cs2) sum_i w_i phi(x + e_i) e_i, all colours of a neighbour
    // from its vectors
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      float v[N];
      comp_load<N>(phi, NN, static_cast<size_t>(wrapn(y + ey(i), ny)) * nx + wrapn(x + ex(i), nx), 0, v);
      const float w3 = 3.0f * (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        gx[k] += w3 * ex(i) * v[k];
        gy[k] += w3 * ey(i) * v[k];
      }
    }
    const float rho = rho_in[n];
    float txx = 0.0f, txy = 0.0f, tyy = 0.0f;
    // V_k = sum_{l != k} beta_kl (rho_k rho_l / rho) n_kl, n_lk = -n_kl
    float Vx[N], Vy[N];
#pragma unroll
    for (int k = 0; k < N; ++k) Vx[k] = Vy[k] = 0.0f;
    int q = 0;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int l = k + 1; l < N; ++l, ++q) {
        const float Gx = ph[l] * gx[k] - ph[k] * gx[l];  // G_kl = phi_l grad phi_k - phi_k grad phi_l
        const float Gy = ph[l] * gy[k] - ph[k] * gy[l];
        const float g2 = Gx * Gx + Gy * Gy;
        float nxv = 0.0f, nyv = 0.0f;
        if (g2 > 1e-30f) {
          const float rm = rsqrtf(g2);  // 1/|G|
          const float mag = g2 * rm;
          const float pp = ph[k] * ph[l];
          const float ck = fminf(a.cpair[q] * pp * rho * rho, 1.0f);  // Eq. 15
          const float sc = a.sigma[q] * ck * rm;                      // sigma C |G| (I - n n) = sigma C (|G|^2 I - G G)/|G|
          txx += sc * Gy * Gy;
          txy -= sc * Gx * Gy;
          tyy += sc * Gx * Gx;
          const float inv = 1.0f / fmaxf(mag, a.ndelta * pp);
          nxv = Gx * inv;
          nyv = Gy * inv;
        }
        // the segregation parameter of the pair (beta_kl above)
        float b = 1.0f;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          if (m == k || m == l) continue;
          b += fminf(a.beta_A * ph[k] * ph[l] * ph[m], 1.0f) * a.gjunc[q][m];
        }
        const float amp = a.beta0 * b * ph[k] * ph[l] * rho;
        Vx[k] += amp * nxv;
        Vy[k] += amp * nyv;
        Vx[l] -= amp * nxv;
        Vy[l] -= amp * nyv;
      }
    T[n] = make_float4(txx, txy, tyy, 0.0f);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      Vout[static_cast<size_t>(k) * NN + n] = Vx[k];
      Vout[static_cast<size_t>(N + k) * NN + n] = Vy[k];
    }
  }
}

template <int N, bool RED>
__global__ void __launch_bounds__(kNThreads) n_collide_kernel(const float* __restrict__ phi,
                                                              const float* __restrict__ rho_in,
                                                              const float* __restrict__ fi,
                                                              const float4* __restrict__ T,
                                                              const float* __restrict__ Vin, float* __restrict__ fout,
                                                              NArgs a) {
  pdl_wait_then_release();
  const int nx = a.nx, ny = a.ny;
  const size_t NN = static_cast<size_t>(nx) * ny;
  {
    // one row per block row of the grid: no division for the node's coordinates
    const int y = static_cast<int>(blockIdx.x);
    const int x = static_cast<int>(blockIdx.y) * kNThreads + static_cast<int>(threadIdx.x);
    if (x >= nx) return;
    const size_t n = static_cast<size_t>(y) * nx + x;
    // F_s = div T (Eq. 11), each component by Eq. fd1
    float Fx = 0.0f, Fy = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const size_t m = static_cast<size_t>(wrapn(y + ey(i), ny)) * nx + wrapn(x + ex(i), nx);
      const float w3 = 3.0f * (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
      const float4 t = T[m];
      const float txx = t.x, txy = t.y, tyy = t.z;
      Fx += w3 * (ex(i) * txx + ey(i) * txy);
      Fy += w3 * (ex(i) * txy + ey(i) * tyy);
    }
    const float rho = rho_in[n];
    float ph[N];
    comp_load<N>(phi, NN, n, 0, ph);
    float f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fi[static_cast<size_t>(i) * NN + n];
    float mx = 0.0f, my = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      mx += ex(i) * f[i];
      my += ey(i) * f[i];
    }
    const float irho = 1.0f / rho;
    const float ux = (mx + 0.5f * Fx) * irho, uy = (my + 0.5f * Fy) * irho;  // Eq. uk1
    float inu = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) inu += ph[k] * a.inv_nu[k];  // rho/nu = sum_k rho_k/nu_k
    const float om = inu / (3.0f + 0.5f * inu);               // 1/tau_f, tau_f = 3 nu + 1/2
    const float g = 1.0f - 0.5f * om;                         // Guo prefactor 1 - 1/(2 tau_f)
    const float uu = ux * ux + uy * uy;
    float fd[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float eu = ex(i) * ux + ey(i) * uy;
      const float feq = wt(i) * rho * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);  // Eq. 3
      const float cx = 3.0f * (ex(i) - ux) + 9.0f * eu * ex(i);
      const float cy = 3.0f * (ey(i) - uy) + 9.0f * eu * ey(i);
      const float Phi = wt(i) * g * (cx * Fx + cy * Fy);                               // Eq. 5
      fd[i] = f[i] + om * (feq - f[i]) + Phi;                                          // Eqs. 1, 2
    }
    // the recolouring vectors V_k of the tension kernel
    float Vx[N], Vy[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      Vx[k] = Vin[static_cast<size_t>(k) * NN + n];
      Vy[k] = Vin[static_cast<size_t>(N + k) * NN + n];
    }
    // Eq. 6, stored at the node (the next step's pull streams it, Eq. 30), as
    // 9 N populations or as the reduced state
    if constexpr (RED) {
      comp_store<N>(fout, NN, n, 0, ph);
      comp_store<N>(fout, NN, n, 1, Vx);
      comp_store<N>(fout, NN, n, 2, Vy);
      float* __restrict__ fdo = fout + kRedVec<N> * NN;
#pragma unroll
      for (int i = 0; i < 9; ++i) fdo[static_cast<size_t>(i) * NN + n] = fd[i];
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k)
#pragma unroll
        for (int i = 0; i < 9; ++i)
          fout[(static_cast<size_t>(k) * 9 + i) * NN + n] = recolour2(ph[k], fd[i], a.wrec[i], edot2(i, Vx[k], Vy[k]));
    }
  }
}

// the reduced state g expanded into the populations it stands for, stored at
// the producing node
template <int N>
__global__ void __launch_bounds__(kNThreads) n_expand_kernel(const float* __restrict__ g, float* __restrict__ f,
                                                             NArgs a) {
  const int nx = a.nx, ny = a.ny;
  const size_t NN = static_cast<size_t>(nx) * ny;
  const int y = static_cast<int>(blockIdx.x);
  const int x = static_cast<int>(blockIdx.y) * kNThreads + static_cast<int>(threadIdx.x);
  if (x >= nx) return;
  const size_t n = static_cast<size_t>(y) * nx + x;
  float ph[N], Vx[N], Vy[N];
  comp_load<N>(g, NN, n, 0, ph);
  comp_load<N>(g, NN, n, 1, Vx);
  comp_load<N>(g, NN, n, 2, Vy);
  const float* __restrict__ fd = g + kRedVec<N> * NN;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float fdi = fd[static_cast<size_t>(i) * NN + n];
#pragma unroll
    for (int k = 0; k < N; ++k)
      f[(static_cast<size_t>(k) * 9 + i) * NN + n] = recolour2(ph[k], fdi, a.wrec[i], edot2(i, Vx[k], Vy[k]));
  }
}

// Observables of the state the density and tension kernels have just
// processed: rho_k = phi_k rho, u = (sum_i f_i e_i + F/2) / rho (Eq. uk1, F
// by Eq. fd1 from the tension tensor), p = rho / 3, FP64 (any may be null)
template <int N>
__global__ void __launch_bounds__(kNThreads) n_fields_kernel(const float* __restrict__ phi,
                                                             const float* __restrict__ rho_in,
                                                             const float* __restrict__ fi,
                                                             const float4* __restrict__ T, double* __restrict__ rho_out,
                                                             double* __restrict__ ux_out, double* __restrict__ uy_out,
                                                             double* __restrict__ p_out, NArgs a) {
  const int nx = a.nx, ny = a.ny;
  const size_t NN = static_cast<size_t>(nx) * ny;
  const int y = static_cast<int>(blockIdx.x);
  const int x = static_cast<int>(blockIdx.y) * kNThreads + static_cast<int>(threadIdx.x);
  if (x >= nx) return;
  const size_t n = static_cast<size_t>(y) * nx + x;
  const float rho = rho_in[n];
  if (rho_out) {
    float ph[N];
    comp_load<N>(phi, NN, n, 0, ph);
#pragma unroll
    for (int k = 0; k < N; ++k) rho_out[static_cast<size_t>(k) * NN + n] = static_cast<double>(ph[k] * rho);
  }
  if (ux_out || uy_out) {
    float Fx = 0.0f, Fy = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const size_t m = static_cast<size_t>(wrapn(y + ey(i), ny)) * nx + wrapn(x + ex(i), nx);
      const float w3 = 3.0f * (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
      const float4 t = T[m];
      const float txx = t.x, txy = t.y, tyy = t.z;
      Fx += w3 * (ex(i) * txx + ey(i) * txy);
      Fy += w3 * (ex(i) * txy + ey(i) * tyy);
    }
    float mx = 0.0f, my = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const float fv = fi[static_cast<size_t>(i) * NN + n];
      mx += ex(i) * fv;
      my += ey(i) * fv;
    }
    const float irho = 1.0f / rho;
    if (ux_out) ux_out[n] = static_cast<double>((mx + 0.5f * Fx) * irho);
    if (uy_out) uy_out[n] = static_cast<double>((my + 0.5f * Fy) * irho);
  }
  if (p_out) p_out[n] = static_cast<double>(rho) / 3.0;
}

int grid_of(size_t NN) {
  size_t g = (NN + kNThreads - 1) / kNThreads;
  return static_cast<int>(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

// one step from the state fin (populations, or the reduced state with
// in_red) to fout (the reduced state with out_red)
template <int N>
cudaError_t n_step(const float* fin, float* fout, float* work, const NArgs& a, cudaStream_t s, bool in_red,
                   bool out_red) {
  const size_t NN = static_cast<size_t>(a.nx) * a.ny;
  // the tension tensor first (one float4 per node), then the fractions (kCK
  // vector planes of kCW floats), so that both are aligned for vector access
  float4* T = reinterpret_cast<float4*>(work);
  float* phi = work + 4 * NN;
  float* rho = phi + kRedVec<N> / 3 * NN;
  float* fi = rho + NN;
  float* V = fi + 9 * NN;
  const dim3 g(static_cast<unsigned>(a.ny), static_cast<unsigned>((a.nx + kNThreads - 1) / kNThreads));
  const dim3 b(kNThreads);
  cudaError_t e = in_red ? launch_pdl(n_density_kernel<N, true>, g, b, s, fin, phi, rho, fi, a)
                         : launch_pdl(n_density_kernel<N, false>, g, b, s, fin, phi, rho, fi, a);
  if (e == cudaSuccess) e = launch_pdl(n_tension_kernel<N>, g, b, s, phi, rho, T, V, a);
  if (e == cudaSuccess)
    e = out_red ? launch_pdl(n_collide_kernel<N, true>, g, b, s, phi, rho, fi, T, V, fout, a)
                : launch_pdl(n_collide_kernel<N, false>, g, b, s, phi, rho, fi, T, V, fout, a);
  return e;
}

template <int N, bool RED>
cudaError_t n_fields(const float* fin, float* work, double* rho, double* ux, double* uy, double* p, const NArgs& a,
                     cudaStream_t s) {
  const size_t NN = static_cast<size_t>(a.nx) * a.ny;
  float4* T = reinterpret_cast<float4*>(work);
  float* phi = work + 4 * NN;
  float* rh = phi + kRedVec<N> / 3 * NN;
  float* fi = rh + NN;
  float* V = fi + 9 * NN;
  const dim3 g(static_cast<unsigned>(a.ny), static_cast<unsigned>((a.nx + kNThreads - 1) / kNThreads));
  n_density_kernel<N, RED><<<g, kNThreads, 0, s>>>(fin, phi, rh, fi, a);
  n_tension_kernel<N><<<g, kNThreads, 0, s>>>(phi, rh, T, V, a);
  n_fields_kernel<N><<<g, kNThreads, 0, s>>>(phi, rh, fi, T, rho, ux, uy, p, a);
  return cudaGetLastError();
}

template <int N>
cudaError_t n_fields_red(bool red, const float* fin, float* work, double* rho, double* ux, double* uy, double* p,
                         const NArgs& a, cudaStream_t s) {
  return red ? n_fields<N, true>(fin, work, rho, ux, uy, p, a, s) : n_fields<N, false>(fin, work, rho, ux, uy, p, a, s);
}

cudaError_t n_fields_any(int N, bool red, const float* fin, float* work, double* rho, double* ux, double* uy,
                         double* p, const NArgs& a, cudaStream_t s) {
  switch (N) {
    case 2: return n_fields_red<2>(red, fin, work, rho, ux, uy, p, a, s);
    case 3: return n_fields_red<3>(red, fin, work, rho, ux, uy, p, a, s);
    case 4: return n_fields_red<4>(red, fin, work, rho, ux, uy, p, a, s);
    case 5: return n_fields_red<5>(red, fin, work, rho, ux, uy, p, a, s);
    case 6: return n_fields_red<6>(red, fin, work, rho, ux, uy, p, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t n_step_any(int N, const float* fin, float* fout, float* work, const NArgs& a, cudaStream_t s, bool in_red,
                       bool out_red) {
  switch (N) {
    case 2: return n_step<2>(fin, fout, work, a, s, in_red, out_red);
    case 3: return n_step<3>(fin, fout, work, a, s, in_red, out_red);
    case 4: return n_step<4>(fin, fout, work, a, s, in_red, out_red);
    case 5: return n_step<5>(fin, fout, work, a, s, in_red, out_red);
    case 6: return n_step<6>(fin, fout, work, a, s, in_red, out_red);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t n_expand_any(int N, const float* g, float* f, const NArgs& a, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>(a.ny), static_cast<unsigned>((a.nx + kNThreads - 1) / kNThreads));
  switch (N) {
    case 2: n_expand_kernel<2><<<grid, kNThreads, 0, s>>>(g, f, a); break;
    case 3: n_expand_kernel<3><<<grid, kNThreads, 0, s>>>(g, f, a); break;
    case 4: n_expand_kernel<4><<<grid, kNThreads, 0, s>>>(g, f, a); break;
    case 5: n_expand_kernel<5><<<grid, kNThreads, 0, s>>>(g, f, a); break;
    case 6: n_expand_kernel<6><<<grid, kNThreads, 0, s>>>(g, f, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// intermediates, rounded up to 64 floats so that the FP64 staging behind them
// is aligned
size_t work_floats(int N, size_t NN) {
  const size_t phiv = N <= 2 ? 2 : (N <= 4 ? 4 : 8);  // the fractions as vectors of 2 or 4 floats
  return ((4 + phiv + 1 + 9 + static_cast<size_t>(2) * N) * NN + 63) / 64 * 64;
}

// stored (post-collision, at the producing node) <-> post-streaming populations
__global__ void n_set_kernel(const double* __restrict__ fpost, float* __restrict__ f, int nx, int ny, int planes) {
  const size_t NN = static_cast<size_t>(nx) * ny;
  const int p = blockIdx.y;  // k*9 + i
  const int i = p % 9;
  for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < NN;
       n += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(n % nx), y = static_cast<int>(n / nx);
    // stored(x) = post-streaming(x + e_i)
    const size_t src = static_cast<size_t>(wrapn(y + ey(i), ny)) * nx + wrapn(x + ex(i), nx);
    f[static_cast<size_t>(p) * NN + n] = static_cast<float>(fpost[static_cast<size_t>(p) * NN + src]);
  }
  (void)planes;
}

// rest equilibrium per colour from the densities, in the stored form:
// stored(x) = post-streaming(x + e_i) = w_i rho_k(x + e_i); one block row
// per colour x direction plane
__global__ void n_init_kernel(const double* __restrict__ rho, float* __restrict__ f, int nx, int ny) {
  const size_t NN = static_cast<size_t>(nx) * ny;
  const int p = blockIdx.y;  // k*9 + i
  const int k = p / 9, i = p % 9;
  const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < NN;
       n += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(n % nx), y = static_cast<int>(n / nx);
    const size_t src = static_cast<size_t>(wrapn(y + ey(i), ny)) * nx + wrapn(x + ex(i), nx);
    f[static_cast<size_t>(p) * NN + n] = static_cast<float>(w * rho[static_cast<size_t>(k) * NN + src]);
  }
}

__global__ void n_get_kernel(const float* __restrict__ f, double* __restrict__ fpost, int nx, int ny) {
  const size_t NN = static_cast<size_t>(nx) * ny;
  const int p = blockIdx.y;
  const int i = p % 9;
  for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < NN;
       n += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(n % nx), y = static_cast<int>(n / nx);
    const size_t src = static_cast<size_t>(wrapn(y - ey(i), ny)) * nx + wrapn(x - ex(i), nx);
    fpost[static_cast<size_t>(p) * NN + n] = static_cast<double>(f[static_cast<size_t>(p) * NN + src]);
  }
}

// FP64 per-colour mass and lattice momentum: one block per colour x direction
// plane, a fixed-order tree per block, then a fixed-order sum on the host
__global__ void n_plane_sum_kernel(const float* __restrict__ f, int NNi, double* __restrict__ out) {
  const size_t NN = static_cast<size_t>(NNi);
  const int p = blockIdx.x;
  double s = 0.0;
  for (size_t n = threadIdx.x; n < NN; n += blockDim.x) s += static_cast<double>(f[static_cast<size_t>(p) * NN + n]);
  __shared__ double sh[kNThreads];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kNThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[p] = sh[0];
}

double g_of(double X) {  // Eq. 20
  if (X < -1.0) return 1.0;
  if (X < 0.0) return 1.0 - std::sqrt(1.0 - X * X);
  if (X <= 1.0) return std::sqrt(1.0 - X * X) - 1.0;
  return -1.0;
}

}  // namespace
}  // namespace lbm3

struct lbm3n_ctx {
  int N = 0, nx = 0, ny = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  float* buf[2] = {nullptr, nullptr};
  float* work = nullptr;
  double* sums = nullptr;
  int cur = 0;
  bool state_set = false;
  bool reduced = false;  // the storage form of the steps (LBM3_REDUCED)
  bool red = false;      // buf[cur] holds the reduced state (else populations)
  int64_t t = 0;
  lbm3::NArgs args{};
  std::string msg;
};

namespace {

lbm3_status nfail(lbm3n_ctx* c, lbm3_status st, const std::string& m) {
  if (c) c->msg = m;
  return st;
}

lbm3_status ncuda(lbm3n_ctx* c, cudaError_t e, const char* where) {
  return nfail(c, LBM3_ECUDA, std::string("lbm3n: ") + where + ": " + cudaGetErrorString(e));
}

// the current state as stored populations: buf[cur] itself, or the reduced
// state expanded into the idle buffer
const float* stored_populations(lbm3n_ctx* c, cudaError_t* e) {
  *e = cudaSuccess;
  if (!c->red) return c->buf[c->cur];
  *e = lbm3::n_expand_any(c->N, c->buf[c->cur], c->buf[c->cur ^ 1], c->args, c->stream);
  return c->buf[c->cur ^ 1];
}

}  // namespace

extern "C" {

lbm3_status lbm3n_create(const lbm3n_params* p, void* cuda_stream, lbm3n_ctx** out) {
  if (!out) return LBM3_EINVAL;
  *out = nullptr;
  if (!p || !p->tau || !p->rho0 || !p->sigma) return LBM3_EINVAL;
  const int N = p->nfluids;
  if (N < 2 || N > lbm3::kMaxFluids || p->nx < 1 || p->ny < 1) return LBM3_EINVAL;
  if (static_cast<double>(p->nx) * p->ny * 9 * N >= 2147483648.0) return LBM3_EINVAL;
  if (!(p->beta0 > 0.0 && p->beta0 <= 1.0) || p->beta_form < 0 || p->beta_form > 1 || p->recolor_form < 0 ||
      p->recolor_form > 1 || !(p->normal_delta >= 0.0 && p->normal_delta <= 1.0) ||
      (p->storage != LBM3_FP32 && p->storage != LBM3_REDUCED))
    return LBM3_EINVAL;
  for (int k = 0; k < N; ++k) {
    if (!(p->tau[k] > 0.5) || !(p->rho0[k] > 0.0)) return LBM3_EINVAL;
    for (int l = 0; l < N; ++l) {
      const double s = p->sigma[k * N + l], t = p->sigma[l * N + k];
      if (k == l ? s != 0.0 : !(s > 0.0 && s == t)) return LBM3_EINVAL;
    }
  }
  lbm3n_ctx* c = new (std::nothrow) lbm3n_ctx();
  if (!c) return LBM3_ENOMEM;
  c->N = N;
  c->nx = p->nx;
  c->ny = p->ny;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->reduced = p->storage == LBM3_REDUCED;
  cudaGetDevice(&c->device);
  lbm3::NArgs& a = c->args;
  a.nx = p->nx;
  a.ny = p->ny;
  for (int k = 0; k < N; ++k) a.inv_nu[k] = static_cast<float>(3.0 / (p->tau[k] - 0.5));
  for (int k = 0; k < N; ++k)
    for (int l = k + 1; l < N; ++l) {
      const int q = lbm3::pair_index(k, l, N);
      a.sigma[q] = static_cast<float>(p->sigma[k * N + l]);
      a.cpair[q] = static_cast<float>(1e6 / (p->rho0[k] * p->rho0[l]));
      for (int m = 0; m < N; ++m) {
        double gv = 0.0;
        if (m != k && m != l) {
          const double smk = p->sigma[m * N + k], sml = p->sigma[m * N + l], skl = p->sigma[k * N + l];
          gv = lbm3::g_of((smk * smk + sml * sml - skl * skl) / (2.0 * smk * sml));  // Eqs. 18, 20
        }
        a.gjunc[q][m] = static_cast<float>(gv);
      }
    }
  a.beta0 = static_cast<float>(p->beta0);
  a.beta_A = p->beta_form == 0 ? 35.0f : 0.0f;
  for (int i = 0; i < 9; ++i) {
    const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const double len = std::sqrt(static_cast<double>(lbm3::ex(i) * lbm3::ex(i) + lbm3::ey(i) * lbm3::ey(i)));
    a.wrec[i] = static_cast<float>((p->recolor_form == 0 && i != 0) ? w / len : w);
  }
  a.ndelta = static_cast<float>(p->normal_delta);
  const size_t NN = static_cast<size_t>(p->nx) * p->ny;
  const size_t pop = static_cast<size_t>(9) * N * NN * sizeof(float);
  void *b0 = nullptr, *b1 = nullptr, *w = nullptr, *sm = nullptr;
  if (cudaMalloc(&b0, pop) != cudaSuccess || cudaMalloc(&b1, pop) != cudaSuccess ||
      cudaMalloc(&w, lbm3::work_floats(N, NN) * sizeof(float) + 9 * N * NN * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sm, 9 * N * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (b0) cudaFree(b0);
    if (b1) cudaFree(b1);
    if (w) cudaFree(w);
    delete c;
    return LBM3_ENOMEM;
  }
  c->buf[0] = static_cast<float*>(b0);
  c->buf[1] = static_cast<float*>(b1);
  c->work = static_cast<float*>(w);
  c->sums = static_cast<double*>(sm);
  *out = c;
  return LBM3_OK;
}

lbm3_status lbm3n_set_populations(lbm3n_ctx* c, const double* f, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!f) return nfail(c, LBM3_EINVAL, "lbm3n_set_populations: NULL f");
  const size_t NN = static_cast<size_t>(c->nx) * c->ny;
  const size_t bytes = static_cast<size_t>(9) * c->N * NN * sizeof(double);
  const double* src = f;
  // FP64 staging behind the intermediates in the work allocation
  double* staging = reinterpret_cast<double*>(c->work + lbm3::work_floats(c->N, NN));
  if (!on_device) {
    cudaError_t e = cudaMemcpyAsync(staging, f, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return ncuda(c, e, "copy to the device");
    src = staging;
  }
  dim3 grid(lbm3::grid_of(NN), 9 * c->N);
  lbm3::n_set_kernel<<<grid, lbm3::kNThreads, 0, c->stream>>>(src, c->buf[c->cur], c->nx, c->ny, 9 * c->N);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return ncuda(c, e, "lbm3n_set_populations");
  c->state_set = true;
  c->red = false;
  c->t = 0;
  return LBM3_OK;
}

lbm3_status lbm3n_init(lbm3n_ctx* c, const double* rho, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!rho || on_device) return nfail(c, LBM3_EINVAL, "lbm3n_init: host densities rho[N][ny][nx] required");
  const size_t NN = static_cast<size_t>(c->nx) * c->ny;
  for (size_t n = 0; n < static_cast<size_t>(c->N) * NN; ++n)
    if (!(rho[n] >= 0.0)) return nfail(c, LBM3_EINVAL, "lbm3n_init: rho_k must be >= 0");
  // the densities go through the FP64 staging area (N of its 9 N planes)
  double* staging = reinterpret_cast<double*>(c->work + lbm3::work_floats(c->N, NN));
  cudaError_t e = cudaMemcpyAsync(staging, rho, static_cast<size_t>(c->N) * NN * sizeof(double),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    lbm3::n_init_kernel<<<dim3(lbm3::grid_of(NN), 9 * c->N), lbm3::kNThreads, 0, c->stream>>>(
        staging, c->buf[c->cur], c->nx, c->ny);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return ncuda(c, e, "lbm3n_init");
  c->state_set = true;
  c->red = false;
  c->t = 0;
  return LBM3_OK;
}

lbm3_status lbm3n_step(lbm3n_ctx* c, int64_t n) {
  if (!c) return LBM3_EINVAL;
  if (n < 0) return nfail(c, LBM3_EINVAL, "lbm3n_step: n < 0");
  if (!c->state_set) return nfail(c, LBM3_ESTATE, "lbm3n_step: state not set");
  for (int64_t s = 0; s < n; ++s) {
    const cudaError_t e = lbm3::n_step_any(c->N, c->buf[c->cur], c->buf[c->cur ^ 1], c->work, c->args, c->stream,
                                           c->red, c->reduced);
    if (e != cudaSuccess) return ncuda(c, e, "lbm3n_step");
    c->cur ^= 1;
    c->red = c->reduced;
    c->t += 1;
  }
  return LBM3_OK;
}

lbm3_status lbm3n_populations(lbm3n_ctx* c, double* f, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!f) return nfail(c, LBM3_EINVAL, "lbm3n_populations: NULL f");
  if (!c->state_set) return nfail(c, LBM3_ESTATE, "lbm3n_populations: state not set");
  const size_t NN = static_cast<size_t>(c->nx) * c->ny;
  double* dst = on_device ? f : reinterpret_cast<double*>(c->work + lbm3::work_floats(c->N, NN));
  dim3 grid(lbm3::grid_of(NN), 9 * c->N);
  cudaError_t e;
  const float* src = stored_populations(c, &e);
  if (e == cudaSuccess) {
    lbm3::n_get_kernel<<<grid, lbm3::kNThreads, 0, c->stream>>>(src, dst, c->nx, c->ny);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(f, dst, static_cast<size_t>(9) * c->N * NN * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return ncuda(c, e, "lbm3n_populations");
  return LBM3_OK;
}

lbm3_status lbm3n_fields(lbm3n_ctx* c, double* rho, double* ux, double* uy, double* p, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!c->state_set) return nfail(c, LBM3_ESTATE, "lbm3n_fields: state not set");
  const size_t NN = static_cast<size_t>(c->nx) * c->ny;
  // the FP64 staging area holds the host case's outputs: N + 3 of its 9 N planes
  double* staging = reinterpret_cast<double*>(c->work + lbm3::work_floats(c->N, NN));
  double* d_rho = rho ? (on_device ? rho : staging) : nullptr;
  double* d_ux = ux ? (on_device ? ux : staging + static_cast<size_t>(c->N) * NN) : nullptr;
  double* d_uy = uy ? (on_device ? uy : staging + static_cast<size_t>(c->N + 1) * NN) : nullptr;
  double* d_p = p ? (on_device ? p : staging + static_cast<size_t>(c->N + 2) * NN) : nullptr;
  cudaError_t e =
      lbm3::n_fields_any(c->N, c->red, c->buf[c->cur], c->work, d_rho, d_ux, d_uy, d_p, c->args, c->stream);
  if (e == cudaSuccess && !on_device) {
    if (rho)
      e = cudaMemcpyAsync(rho, d_rho, static_cast<size_t>(c->N) * NN * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess && ux) e = cudaMemcpyAsync(ux, d_ux, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && uy) e = cudaMemcpyAsync(uy, d_uy, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, d_p, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return ncuda(c, e, "lbm3n_fields");
  return LBM3_OK;
}

lbm3_status lbm3n_mass(lbm3n_ctx* c, double* mass, double* mom) {
  if (!c) return LBM3_EINVAL;
  if (!c->state_set) return nfail(c, LBM3_ESTATE, "lbm3n_mass: state not set");
  const size_t NN = static_cast<size_t>(c->nx) * c->ny;
  cudaError_t e;
  const float* src = stored_populations(c, &e);
  if (e == cudaSuccess) {
    lbm3::n_plane_sum_kernel<<<9 * c->N, lbm3::kNThreads, 0, c->stream>>>(src, static_cast<int>(NN), c->sums);
    e = cudaGetLastError();
  }
  std::vector<double> h(static_cast<size_t>(9) * c->N);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), c->sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return ncuda(c, e, "lbm3n_mass");
  double mx = 0.0, my = 0.0;
  for (int k = 0; k < c->N; ++k) {
    double m = 0.0;
    for (int i = 0; i < 9; ++i) {
      const double v = h[static_cast<size_t>(k) * 9 + i];
      m += v;
      mx += lbm3::ex(i) * v;
      my += lbm3::ey(i) * v;
    }
    if (mass) mass[k] = m;
  }
  if (mom) {
    mom[0] = mx;
    mom[1] = my;
  }
  return LBM3_OK;
}

lbm3_status lbm3n_destroy(lbm3n_ctx* c) {
  if (!c) return LBM3_OK;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->buf[0]);
  cudaFree(c->buf[1]);
  cudaFree(c->work);
  cudaFree(c->sums);
  cudaGetLastError();
  delete c;
  return LBM3_OK;
}

const char* lbm3n_last_error(const lbm3n_ctx* c) { return c ? c->msg.c_str() : "lbm3n: NULL context"; }

}  // extern "C"
