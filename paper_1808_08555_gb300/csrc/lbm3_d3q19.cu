// N-fluid colour-gradient step on the D3Q19 lattice (arXiv 1808.08555: the
// model of Sec. 2 is written in vector form, Eq. fd1, Eq. 11 and the
// recolouring of Eq. 6 hold in any dimension; the paper simulates two
// dimensions).  A first CUDA path for 2 <= N <= kMaxFluids3, three kernels
// per step over global-memory intermediates, one node per thread, on
// (x-block, y, z) grids:
//   densities:  pull the 19N populations (Eq. 30), rho_k, rho, phi_k (the
//               largest fraction as the complement of the others), the total
//               distribution f_i
//   tension:    grad phi_k (Eq. fd1 on D3Q19), G_kl and C_kl (Eq. 15) for the
//               N(N-1)/2 pairs, the 3x3 tension tensor of Eq. 11 summed over
//               the pairs, the recolouring normals G / max(|G|, delta phi_k phi_l)
//   collide:    F_s = div T (Eq. fd1), u (Eq. uk1), tau_f (Eqs. vis_1, tau),
//               BGK with Guo's forcing (Eqs. 1-3, 5), beta_kl, recolouring
//               (Eq. 6); f^ddagger stored at the node that produced it
// beta_kl as for the two-dimensional N-fluid path (Eq. 19 for N = 3, one
// junction term per third fluid beyond), g(X_kl^m) precomputed on the host.
//
// Lattice: rest (weight 1/3), the six axis vectors (1/18), the twelve edge
// diagonals (1/36), c_s^2 = 1/3, opposite directions adjacent:
//   0 (0,0,0)  1 (1,0,0)  2 (-1,0,0)  3 (0,1,0)  4 (0,-1,0)  5 (0,0,1)  6 (0,0,-1)
//   7 (1,1,0)  8 (-1,-1,0)  9 (1,-1,0)  10 (-1,1,0)  11 (1,0,1)  12 (-1,0,-1)
//   13 (1,0,-1)  14 (-1,0,1)  15 (0,1,1)  16 (0,-1,-1)  17 (0,1,-1)  18 (0,-1,1)
// Layout: populations [N][19][nz][ny][nx] FP32, unpadded, periodic by index
// arithmetic.  Intermediates, node-major where a stencil gathers them (one
// vector load per neighbour): the colour fractions and density as one float4
// per node (phi_1, phi_2, phi_3 or 0, rho) for N <= 3, two for N = 4
// ((phi_1 .. phi_4), (rho, 0, 0, 0)); the tension tensor as a float4 (xx, xy,
// xz, yy) and a float2 (yz, zz) per node; then planes f_i [19] and normals
// [P][3] with P = N(N-1)/2, each [nz][ny][nx].

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

constexpr int kMaxFluids3 = 4;
constexpr int kMaxPairs3 = kMaxFluids3 * (kMaxFluids3 - 1) / 2;
constexpr int Q3 = 19;
constexpr int kBX = 128;  // threads per block, along x

__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}
__host__ __device__ constexpr double w3d(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
// FP32 weights whose exact sum is 1 (1/36 rounded down to an even multiple of
// its ulp, 1/18 twice that, 1/3 the remainder, within 2 ulp of each): with
// the nearest floats the sum is 1 + 1.5e-8 and every collision would create
// that fraction of mass (2.5e-8 per step at tau = 0.6)
__host__ __device__ constexpr float w3f(int i) {
  return i == 0 ? 0x1.555558p-2f : (i < 7 ? 0x1.c71c70p-5f : 0x1.c71c70p-6f);
}

struct DArgs {
  int nx, ny, nz;
  float inv_nu[kMaxFluids3];            // 1/nu_k
  float sigma[kMaxPairs3];              // sigma_kl for pairs k < l in row order
  float cpair[kMaxPairs3];              // 1e6 / (rho0_k rho0_l)
  float gjunc[kMaxPairs3][kMaxFluids3];  // g(X_kl^m) (0 for m = k, l)
  float beta0, beta_A;                  // beta_A = 35 (0: Eq. fu, constant beta)
  float wrec[Q3];                       // recolouring weights w_i / |e_i| or w_i
  float ndelta;
};

__host__ __device__ constexpr int pair3(int k, int l, int n) {  // k < l
  return k * n - k * (k + 1) / 2 + (l - k - 1);
}

__device__ __forceinline__ int wrap3(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

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

// the node of this thread and the strides of the [nz][ny][nx] planes
struct Node {
  int x, y, z;
  size_t n, NN;
};
__device__ __forceinline__ bool node_of(const DArgs& a, Node* o) {
  o->x = static_cast<int>(blockIdx.x) * kBX + static_cast<int>(threadIdx.x);
  o->y = static_cast<int>(blockIdx.y);
  o->z = static_cast<int>(blockIdx.z);
  o->NN = static_cast<size_t>(a.nx) * a.ny * a.nz;
  o->n = (static_cast<size_t>(o->z) * a.ny + o->y) * a.nx + o->x;
  return o->x < a.nx;
}
// index of the node at offset (dx, dy, dz), periodic
__device__ __forceinline__ size_t at(const DArgs& a, const Node& p, int dx, int dy, int dz) {
  return (static_cast<size_t>(wrap3(p.z + dz, a.nz)) * a.ny + wrap3(p.y + dy, a.ny)) * a.nx + wrap3(p.x + dx, a.nx);
}

// float4 per node of the (phi_k, rho) array
template <int N>
constexpr int kPRV = N <= 3 ? 1 : 2;

template <int N>
__device__ __forceinline__ void pr_store(float4* __restrict__ pr, size_t n, const float (&ph)[N], float rho) {
  if constexpr (N == 2) {
    pr[n] = make_float4(ph[0], ph[1], 0.0f, rho);
  } else if constexpr (N == 3) {
    pr[n] = make_float4(ph[0], ph[1], ph[2], rho);
  } else {
    pr[2 * n] = make_float4(ph[0], ph[1], ph[2], ph[3]);
    pr[2 * n + 1] = make_float4(rho, 0.0f, 0.0f, 0.0f);
  }
}
// the N colour fractions of node n (one vector load for any N <= 4)
template <int N>
__device__ __forceinline__ void pr_phi(const float4* __restrict__ pr, size_t n, float (&ph)[N]) {
  const float4 v = pr[n * kPRV<N>];
  ph[0] = v.x;
  ph[1] = v.y;
  if constexpr (N >= 3) ph[2] = v.z;
  if constexpr (N >= 4) ph[3] = v.w;
}
template <int N>
__device__ __forceinline__ float pr_rho(const float4* __restrict__ pr, size_t n) {
  if constexpr (N <= 3) return pr[n].w;
  return pr[2 * n + 1].x;
}

// ------------------------------------------------------------ node level
// The arithmetic of one node, the neighbours' intermediates through
// accessors.

// colour fractions from the colour densities r_k (the largest as the
// complement of the others, so that they sum to 1 exactly) and the density
template <int N>
__device__ __forceinline__ void fractions(const float (&r)[N], float (&ph)[N], float& rho) {
  float rmax = -1.0f;
  int kmax = 0;
  rho = 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    rho += r[k];
    if (r[k] > rmax) {
      rmax = r[k];
      kmax = k;
    }
  }
  const float ir = 1.0f / rho;
  float rest = 1.0f;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (k != kmax) {
      ph[k] = r[k] * ir;
      rest -= ph[k];
    }
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (k == kmax) ph[k] = rest;
}

// The pull (Eq. 30) at node p from stored populations: colour fractions,
// density, and the total distribution f_i = sum_k f_{i,k}
template <int N>
__device__ __forceinline__ void density_node(const float* __restrict__ f, const DArgs& a, const Node& p,
                                             float (&ph)[N], float& rho, float (&tot)[Q3]) {
  const size_t NN = p.NN;
  float r[N];
#pragma unroll
  for (int i = 0; i < Q3; ++i) tot[i] = 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    // a colour's 19 pulled values loaded together, then summed
    float v[Q3];
#pragma unroll
    for (int i = 0; i < Q3; ++i) v[i] = f[(static_cast<size_t>(k) * Q3 + i) * NN + at(a, p, -cx(i), -cy(i), -cz(i))];
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < Q3; ++i) {
      s += v[i];
      tot[i] += v[i];
    }
    r[k] = s;
  }
  fractions<N>(r, ph, rho);
}

// ---------------------------------------------------------- reduced state
// Collision (Eqs. 1-3, 5) uses only the total distribution and the colour
// densities, and the recolouring of Eq. 6 writes
//   f^ddagger_{i,k} = phi_k f^dagger_i + w'_i e_i . V_k,
//   V_k = sum_{l != k} beta_kl (rho_k rho_l / rho) n_kl,
// so a node's 19 N outputs are fixed by phi_k, f^dagger_i and V_k: 19 + 4 N
// values (31 instead of 57 for three fluids).  Layout inside a population
// buffer, by component: four vector planes [nz][ny][nx] of kCW3 floats
// (float2 for N = 2, float4 above) holding the fractions phi_1..N, the x
// components V_1x..V_Nx, the y and the z components, then the float planes
// f^dagger_i.  A pull from direction i loads the source's fractions and only
// the components that e_i has.  For N = 3 the fourth slot of the four vector
// planes holds f^dagger of directions 0, 1, 3 and 5 (whose pulls load that
// plane anyway), and 15 float planes the others.  All N vectors V_k are kept
// although they sum to zero, so that every population is rebuilt from exactly
// the values the collision used.

// e_i . V over the nonzero components of e_i (at most two on D3Q19)
__device__ __forceinline__ float edot(int i, float vx, float vy, float vz) {
  const float a = cx(i) > 0 ? vx : -vx;
  const float b = cy(i) > 0 ? vy : -vy;
  const float c = cz(i) > 0 ? vz : -vz;
  if (cx(i) != 0) return cy(i) != 0 ? __fadd_rn(a, b) : (cz(i) != 0 ? __fadd_rn(a, c) : a);
  if (cy(i) != 0) return cz(i) != 0 ? __fadd_rn(b, c) : b;
  return cz(i) != 0 ? c : 0.0f;
}

// Eq. 6 for one population, f^ddagger = phi_k f^dagger_i + w'_i (e_i . V_k),
// in explicitly rounded operations: the collision's store and the reduced
// state's rebuild give the same bits
__device__ __forceinline__ float recolour(float phk, float fdi, float wr, float ev) {
  return __fmaf_rn(wr, ev, __fmul_rn(phk, fdi));
}

template <int N>
constexpr int kCW3 = N <= 2 ? 2 : 4;  // floats per vector plane
template <int N>
constexpr bool kSlot3 = N == 3;  // f^dagger of four directions in the spare slots
// the vector plane whose spare slot holds f^dagger_i (N = 3), else -1
__host__ __device__ constexpr int slot3(int i) { return i == 0 ? 0 : (i == 1 ? 1 : (i == 3 ? 2 : (i == 5 ? 3 : -1))); }
template <int N>
__host__ __device__ constexpr bool in_slot3(int i) { return kSlot3<N> && slot3(i) >= 0; }
// the float plane of f^dagger_i (not in a slot)
template <int N>
__host__ __device__ constexpr int fd_plane3(int i) {
  return kSlot3<N> ? i - (i > 0) - (i > 1) - (i > 3) - (i > 5) : i;
}
template <int N>
__device__ __forceinline__ const float* fd_base3(const float* g, size_t NN) {
  return g + static_cast<size_t>(4 * kCW3<N>) * NN;
}

// vector plane c (0: phi, 1..3: V_x, V_y, V_z) of node n: the N values and the
// spare slot
template <int N>
__device__ __forceinline__ void cstore3(float* __restrict__ g, size_t NN, size_t n, int c, const float (&v)[N],
                                        float spare) {
  const size_t m = static_cast<size_t>(c) * NN + n;
  if constexpr (N == 2) {
    reinterpret_cast<float2*>(g)[m] = make_float2(v[0], v[1]);
  } else {
    float e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] = q < N ? v[q % N] : spare;
    reinterpret_cast<float4*>(g)[m] = make_float4(e[0], e[1], e[2], e[3]);
  }
}
template <int N>
__device__ __forceinline__ void cload3(const float* __restrict__ g, size_t NN, size_t n, int c, float (&v)[N],
                                       float& spare) {
  const size_t m = static_cast<size_t>(c) * NN + n;
  if constexpr (N == 2) {
    const float2 w = reinterpret_cast<const float2*>(g)[m];
    v[0] = w.x;
    v[1] = w.y;
    spare = 0.0f;
  } else {
    const float4 w = reinterpret_cast<const float4*>(g)[m];
    const float e[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = e[q];
    spare = e[3];
  }
}

// The pull (Eq. 30) at node p from the reduced state: each population
// rebuilt from its source node x - e_i, then the sums of density_node in the
// same order (so that both state forms give the same bits)
template <int N>
__device__ __forceinline__ void density_node_red(const float* __restrict__ g, const DArgs& a, const Node& p,
                                                 float (&ph)[N], float& rho, float (&tot)[Q3]) {
  const size_t NN = p.NN;
  const float* __restrict__ fd = fd_base3<N>(g, NN);
  float r[N];
#pragma unroll
  for (int k = 0; k < N; ++k) r[k] = 0.0f;
  // the pulled f^dagger_i of the float planes loaded together first, then per
  // direction the source's vector planes (loading several directions' vectors
  // together was slower)
  float fdv[Q3];
#pragma unroll
  for (int i = 0; i < Q3; ++i)
    if (!in_slot3<N>(i))
      fdv[i] = fd[static_cast<size_t>(fd_plane3<N>(i)) * NN + at(a, p, -cx(i), -cy(i), -cz(i))];
#pragma unroll
  for (int i = 0; i < Q3; ++i) {
    const size_t src = at(a, p, -cx(i), -cy(i), -cz(i));
    float sp[N], vx[N], vy[N], vz[N], e[4];
#pragma unroll
    for (int k = 0; k < N; ++k) vx[k] = vy[k] = vz[k] = 0.0f;
    cload3<N>(g, NN, src, 0, sp, e[0]);
    if (cx(i) != 0) cload3<N>(g, NN, src, 1, vx, e[1]);
    if (cy(i) != 0) cload3<N>(g, NN, src, 2, vy, e[2]);
    if (cz(i) != 0) cload3<N>(g, NN, src, 3, vz, e[3]);
    const float fdi = in_slot3<N>(i) ? e[slot3(i) < 0 ? 0 : slot3(i)] : fdv[i];
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const float v = recolour(sp[k], fdi, a.wrec[i], edot(i, vx[k], vy[k], vz[k]));
      r[k] += v;
      t += v;
    }
    tot[i] = t;
  }
  fractions<N>(r, ph, rho);
}

template <int N, bool RED>
__device__ __forceinline__ void density_any(const float* __restrict__ f, const DArgs& a, const Node& p,
                                            float (&ph)[N], float& rho, float (&tot)[Q3]) {
  if constexpr (RED)
    density_node_red<N>(f, a, p, ph, rho, tot);
  else
    density_node<N>(f, a, p, ph, rho, tot);
}

// The tension tensor of Eq. 11 (6 components) and the recolouring normals at
// a node, from its own (phi, rho) and its neighbours' fractions phi_at(i, v);
// each pair's normal is handed to nrm_out(q, nx, ny, nz) as soon as it is
// formed
template <int N, typename PhiAt, typename NrmOut>
__device__ __forceinline__ void tension_node(PhiAt phi_at, const DArgs& a, const float (&ph)[N], float rho,
                                             float4& t4, float2& t2, NrmOut nrm_out) {
  float g[N][3];
#pragma unroll
  for (int k = 0; k < N; ++k) g[k][0] = g[k][1] = g[k][2] = 0.0f;
  // Eq. fd1: (1/cs2) sum_i w_i phi(x + e_i) e_i
#pragma unroll
  for (int i = 1; i < Q3; ++i) {
    float v[N];
    phi_at(i, v);
    const float w3 = 3.0f * w3f(i);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      g[k][0] += w3 * cx(i) * v[k];
      g[k][1] += w3 * cy(i) * v[k];
      g[k][2] += w3 * cz(i) * v[k];
    }
  }
  float txx = 0.0f, txy = 0.0f, txz = 0.0f, tyy = 0.0f, tyz = 0.0f, tzz = 0.0f;
  int q = 0;
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int l = k + 1; l < N; ++l, ++q) {
      // G_kl = phi_l grad phi_k - phi_k grad phi_l
      const float Gx = ph[l] * g[k][0] - ph[k] * g[l][0];
      const float Gy = ph[l] * g[k][1] - ph[k] * g[l][1];
      const float Gz = ph[l] * g[k][2] - ph[k] * g[l][2];
      const float g2 = Gx * Gx + Gy * Gy + Gz * Gz;
      float nv[3] = {0.0f, 0.0f, 0.0f};
      if (g2 > 1e-30f) {
        const float rm = rsqrtf(g2);  // 1/|G|
        const float mag = g2 * rm;
        const float pp = ph[k] * ph[l];
        const float ck = fminf(a.cpair[q] * pp * rho * rho, 1.0f);  // Eq. 15
        // sigma C |G| (I - n n) = sigma C (|G|^2 I - G G) / |G|
        const float sc = a.sigma[q] * ck * rm;
        txx += sc * (Gy * Gy + Gz * Gz);
        tyy += sc * (Gx * Gx + Gz * Gz);
        tzz += sc * (Gx * Gx + Gy * Gy);
        txy -= sc * Gx * Gy;
        txz -= sc * Gx * Gz;
        tyz -= sc * Gy * Gz;
        const float inv = 1.0f / fmaxf(mag, a.ndelta * pp);
        nv[0] = Gx * inv;
        nv[1] = Gy * inv;
        nv[2] = Gz * inv;
      }
      nrm_out(q, nv[0], nv[1], nv[2]);
    }
  t4 = make_float4(txx, txy, txz, tyy);
  t2 = make_float2(tyz, tzz);
}

// F_s = div T (Eq. 11): F_a = (1/cs2) sum_i w_i sum_b e_ib T_ab(x + e_i), the
// neighbours' tensors from t_at(i, ta, tb)
template <typename TAt>
__device__ __forceinline__ void divergence_at(TAt t_at, float (&F)[3]) {
  F[0] = F[1] = F[2] = 0.0f;
#pragma unroll
  for (int i = 1; i < Q3; ++i) {
    const float w3 = 3.0f * w3f(i);
    float4 ta;
    float2 tb;
    t_at(i, ta, tb);
    const float txx = ta.x, txy = ta.y, txz = ta.z, tyy = ta.w, tyz = tb.x, tzz = tb.y;
    F[0] += w3 * (cx(i) * txx + cy(i) * txy + cz(i) * txz);
    F[1] += w3 * (cx(i) * txy + cy(i) * tyy + cz(i) * tyz);
    F[2] += w3 * (cx(i) * txz + cy(i) * tyz + cz(i) * tzz);
  }
}
__device__ __forceinline__ void divergence(const float4* __restrict__ T4, const float2* __restrict__ T2,
                                           const DArgs& a, const Node& p, float (&F)[3]) {
  divergence_at(
      [&](int i, float4& ta, float2& tb) {
        const size_t m = at(a, p, cx(i), cy(i), cz(i));
        ta = T4[m];
        tb = T2[m];
      },
      F);
}

// momentum sum_i f_i e_i of the total distribution
__device__ __forceinline__ void momentum_of(const float (&f)[Q3], float (&m)[3]) {
  m[0] = m[1] = m[2] = 0.0f;
#pragma unroll
  for (int i = 1; i < Q3; ++i) {
    m[0] += cx(i) * f[i];
    m[1] += cy(i) * f[i];
    m[2] += cz(i) * f[i];
  }
}
__device__ __forceinline__ void momentum(const float* __restrict__ fi, size_t n, size_t NN, float (&f)[Q3],
                                         float (&m)[3]) {
#pragma unroll
  for (int i = 0; i < Q3; ++i) f[i] = fi[static_cast<size_t>(i) * NN + n];
  momentum_of(f, m);
}

// Collision (BGK with Guo's forcing, Eqs. 1-3, 5; tau_f of Eqs. vis_1, tau),
// the segregation parameters and the recolouring of Eq. 6, stored at node n
// (the next step's pull streams it, Eq. 30) as 19 N populations or, RED, as
// the reduced state; normals from nrm_at(q, c)
template <int N, bool RED, typename NrmAt>
__device__ __forceinline__ void collide_store(const DArgs& a, const float (&F)[3], const float (&ph)[N], float rho,
                                              const float (&f)[Q3], NrmAt nrm_at, float* __restrict__ fout, size_t n,
                                              size_t NN) {
  float m[3];
  momentum_of(f, m);
  const float irho = 1.0f / rho;
  float u[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = (m[c] + 0.5f * F[c]) * irho;  // Eq. uk1
  float inu = 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) inu += ph[k] * a.inv_nu[k];  // rho/nu = sum_k rho_k/nu_k
  const float om = inu / (3.0f + 0.5f * inu);               // 1/tau_f, tau_f = 3 nu + 1/2
  const float gg = 1.0f - 0.5f * om;                        // Guo prefactor 1 - 1/(2 tau_f)
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  float fd[Q3];
#pragma unroll
  for (int i = 0; i < Q3; ++i) {
    const float eu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
    const float feq = w3f(i) * rho * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);  // Eq. 3
    const float c0 = 3.0f * (cx(i) - u[0]) + 9.0f * eu * cx(i);
    const float c1 = 3.0f * (cy(i) - u[1]) + 9.0f * eu * cy(i);
    const float c2 = 3.0f * (cz(i) - u[2]) + 9.0f * eu * cz(i);
    const float Phi = w3f(i) * gg * (c0 * F[0] + c1 * F[1] + c2 * F[2]);               // Eq. 5
    fd[i] = f[i] + om * (feq - f[i]) + Phi;                                            // Eqs. 1, 2
  }
  // V_k = sum_{l != k} beta_kl (rho_k rho_l / rho) n_kl, with n_lk = -n_kl
  float V[N][3];
#pragma unroll
  for (int k = 0; k < N; ++k) V[k][0] = V[k][1] = V[k][2] = 0.0f;
  int q = 0;
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int l = k + 1; l < N; ++l, ++q) {
      float b = 1.0f;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        if (mm == k || mm == l) continue;
        b += fminf(a.beta_A * ph[k] * ph[l] * ph[mm], 1.0f) * a.gjunc[q][mm];
      }
      const float amp = a.beta0 * b * ph[k] * ph[l] * rho;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float nc = nrm_at(q, c);
        V[k][c] += amp * nc;
        V[l][c] -= amp * nc;
      }
    }
  if constexpr (RED) {
    float vx[N], vy[N], vz[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      vx[k] = V[k][0];
      vy[k] = V[k][1];
      vz[k] = V[k][2];
    }
    cstore3<N>(fout, NN, n, 0, ph, fd[0]);
    cstore3<N>(fout, NN, n, 1, vx, fd[1]);
    cstore3<N>(fout, NN, n, 2, vy, fd[3]);
    cstore3<N>(fout, NN, n, 3, vz, fd[5]);
    float* __restrict__ fdo = fout + static_cast<size_t>(4 * kCW3<N>) * NN;
#pragma unroll
    for (int i = 0; i < Q3; ++i)
      if (!in_slot3<N>(i)) fdo[static_cast<size_t>(fd_plane3<N>(i)) * NN + n] = fd[i];
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int i = 0; i < Q3; ++i)
        fout[(static_cast<size_t>(k) * Q3 + i) * NN + n] =
            recolour(ph[k], fd[i], a.wrec[i], edot(i, V[k][0], V[k][1], V[k][2]));
  }
}

// ------------------------------------------------------- three-kernel path

template <int N, bool RED>
__global__ void __launch_bounds__(kBX) d_density_kernel(const float* __restrict__ f, float4* __restrict__ pr,
                                                        float* __restrict__ fi, DArgs a) {
  pdl_wait_then_release();
  Node p;
  if (!node_of(a, &p)) return;
  float ph[N], rho, tot[Q3];
  density_any<N, RED>(f, a, p, ph, rho, tot);
  pr_store<N>(pr, p.n, ph, rho);
#pragma unroll
  for (int i = 0; i < Q3; ++i) fi[static_cast<size_t>(i) * p.NN + p.n] = tot[i];
}

template <int N>
__global__ void __launch_bounds__(kBX) d_tension_kernel(const float4* __restrict__ pr, float4* __restrict__ T4,
                                                        float2* __restrict__ T2, float* __restrict__ nrm, DArgs a) {
  pdl_wait_then_release();
  Node p;
  if (!node_of(a, &p)) return;
  const size_t NN = p.NN;
  float ph[N];
  pr_phi<N>(pr, p.n, ph);
  const float rho = pr_rho<N>(pr, p.n);
  float4 t4;
  float2 t2;
  tension_node<N>([&](int i, float (&v)[N]) { pr_phi<N>(pr, at(a, p, cx(i), cy(i), cz(i)), v); }, a, ph, rho, t4,
                  t2, [&](int q, float nx, float ny, float nz) {
                    nrm[(static_cast<size_t>(q) * 3) * NN + p.n] = nx;
                    nrm[(static_cast<size_t>(q) * 3 + 1) * NN + p.n] = ny;
                    nrm[(static_cast<size_t>(q) * 3 + 2) * NN + p.n] = nz;
                  });
  T4[p.n] = t4;
  T2[p.n] = t2;
}

template <int N, bool RED>
__global__ void __launch_bounds__(kBX) d_collide_kernel(const float4* __restrict__ pr, const float* __restrict__ fi,
                                                        const float4* __restrict__ T4, const float2* __restrict__ T2,
                                                        const float* __restrict__ nrm, float* __restrict__ fout,
                                                        DArgs a) {
  pdl_wait_then_release();
  Node p;
  if (!node_of(a, &p)) return;
  const size_t NN = p.NN;
  float F[3];
  divergence(T4, T2, a, p, F);
  const float rho = pr_rho<N>(pr, p.n);
  float ph[N];
  pr_phi<N>(pr, p.n, ph);
  float f[Q3];
#pragma unroll
  for (int i = 0; i < Q3; ++i) f[i] = fi[static_cast<size_t>(i) * NN + p.n];
  collide_store<N, RED>(a, F, ph, rho, f, [&](int q, int c) { return nrm[(static_cast<size_t>(q) * 3 + c) * NN + p.n]; },
                        fout, p.n, NN);
}

// the reduced state g expanded into the populations it stands for, stored at
// the producing node (the form the population buffers hold between steps)
template <int N>
__global__ void __launch_bounds__(kBX) d_expand_kernel(const float* __restrict__ g, float* __restrict__ f, DArgs a) {
  Node p;
  if (!node_of(a, &p)) return;
  const size_t NN = p.NN;
  float ph[N], vx[N], vy[N], vz[N], e[4];
  cload3<N>(g, NN, p.n, 0, ph, e[0]);
  cload3<N>(g, NN, p.n, 1, vx, e[1]);
  cload3<N>(g, NN, p.n, 2, vy, e[2]);
  cload3<N>(g, NN, p.n, 3, vz, e[3]);
  const float* __restrict__ fd = fd_base3<N>(g, NN);
#pragma unroll
  for (int i = 0; i < Q3; ++i) {
    const float fdi =
        in_slot3<N>(i) ? e[slot3(i) < 0 ? 0 : slot3(i)] : fd[static_cast<size_t>(fd_plane3<N>(i)) * NN + p.n];
#pragma unroll
    for (int k = 0; k < N; ++k)
      f[(static_cast<size_t>(k) * Q3 + i) * NN + p.n] = recolour(ph[k], fdi, a.wrec[i], edot(i, vx[k], vy[k], vz[k]));
  }
}

// Observables of the state the density and tension kernels have just
// processed: rho_k = phi_k rho, u = (sum_i f_i e_i + F/2) / rho (Eq. uk1),
// p = rho / 3, in FP64 (any output may be null)
template <int N>
__global__ void __launch_bounds__(kBX) d_fields_kernel(const float4* __restrict__ pr, const float* __restrict__ fi,
                                                       const float4* __restrict__ T4, const float2* __restrict__ T2,
                                                       double* __restrict__ rho_out, double* __restrict__ u_out,
                                                       double* __restrict__ p_out, DArgs a) {
  Node p;
  if (!node_of(a, &p)) return;
  const size_t NN = p.NN;
  const float rho = pr_rho<N>(pr, p.n);
  if (rho_out) {
    float ph[N];
    pr_phi<N>(pr, p.n, ph);
#pragma unroll
    for (int k = 0; k < N; ++k) rho_out[static_cast<size_t>(k) * NN + p.n] = static_cast<double>(ph[k] * rho);
  }
  if (u_out) {
    float F[3], f[Q3], m[3];
    divergence(T4, T2, a, p, F);
    momentum(fi, p.n, NN, f, m);
    const float irho = 1.0f / rho;
#pragma unroll
    for (int c = 0; c < 3; ++c) u_out[static_cast<size_t>(c) * NN + p.n] = static_cast<double>((m[c] + 0.5f * F[c]) * irho);
  }
  if (p_out) p_out[p.n] = static_cast<double>(rho) / 3.0;
}

dim3 grid3(const DArgs& a) { return dim3((a.nx + kBX - 1) / kBX, a.ny, a.nz); }

// the intermediates' places in the work area
template <int N>
struct Work {
  float4* pr;
  float4* T4;
  float2* T2;
  float* fi;
  float* nrm;
  Work(float* work, size_t NN) {
    // vector arrays first (16-byte aligned offsets), then the planes
    pr = reinterpret_cast<float4*>(work);
    T4 = pr + kPRV<N> * NN;
    T2 = reinterpret_cast<float2*>(T4 + NN);
    fi = reinterpret_cast<float*>(T2 + NN);
    nrm = fi + Q3 * NN;
  }
};

template <int N, bool RED>
cudaError_t d_fields(const float* fin, float* work, double* rho, double* u, double* pr_out, const DArgs& a,
                     cudaStream_t s) {
  const size_t NN = static_cast<size_t>(a.nx) * a.ny * a.nz;
  const Work<N> w(work, NN);
  const dim3 g = grid3(a);
  d_density_kernel<N, RED><<<g, kBX, 0, s>>>(fin, w.pr, w.fi, a);
  d_tension_kernel<N><<<g, kBX, 0, s>>>(w.pr, w.T4, w.T2, w.nrm, a);
  d_fields_kernel<N><<<g, kBX, 0, s>>>(w.pr, w.fi, w.T4, w.T2, rho, u, pr_out, a);
  return cudaGetLastError();
}

cudaError_t d_fields_any(int N, bool red, const float* fin, float* work, double* rho, double* u, double* p,
                         const DArgs& a, cudaStream_t s) {
  switch (N * 2 + (red ? 1 : 0)) {
    case 4: return d_fields<2, false>(fin, work, rho, u, p, a, s);
    case 5: return d_fields<2, true>(fin, work, rho, u, p, a, s);
    case 6: return d_fields<3, false>(fin, work, rho, u, p, a, s);
    case 7: return d_fields<3, true>(fin, work, rho, u, p, a, s);
    case 8: return d_fields<4, false>(fin, work, rho, u, p, a, s);
    case 9: return d_fields<4, true>(fin, work, rho, u, p, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// one step from the state fin (populations, or the reduced state with
// in_red) to fout (the reduced state with out_red)
template <int N>
cudaError_t d_step(const float* fin, float* fout, float* work, const DArgs& a, cudaStream_t s, bool in_red,
                   bool out_red) {
  const size_t NN = static_cast<size_t>(a.nx) * a.ny * a.nz;
  const Work<N> w(work, NN);
  const dim3 g = grid3(a);
  const dim3 b(kBX);
  cudaError_t e = in_red ? launch_pdl(d_density_kernel<N, true>, g, b, s, fin, w.pr, w.fi, a)
                         : launch_pdl(d_density_kernel<N, false>, g, b, s, fin, w.pr, w.fi, a);
  if (e == cudaSuccess) e = launch_pdl(d_tension_kernel<N>, g, b, s, w.pr, w.T4, w.T2, w.nrm, a);
  if (e == cudaSuccess)
    e = out_red ? launch_pdl(d_collide_kernel<N, true>, g, b, s, w.pr, w.fi, w.T4, w.T2, w.nrm, fout, a)
                : launch_pdl(d_collide_kernel<N, false>, g, b, s, w.pr, w.fi, w.T4, w.T2, w.nrm, fout, a);
  return e;
}

cudaError_t d_step_any(int N, const float* fin, float* fout, float* work, const DArgs& a, cudaStream_t s,
                       bool in_red, bool out_red) {
  switch (N) {
    case 2: return d_step<2>(fin, fout, work, a, s, in_red, out_red);
    case 3: return d_step<3>(fin, fout, work, a, s, in_red, out_red);
    case 4: return d_step<4>(fin, fout, work, a, s, in_red, out_red);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t d_expand_any(int N, const float* g, float* f, const DArgs& a, cudaStream_t s) {
  switch (N) {
    case 2: d_expand_kernel<2><<<grid3(a), kBX, 0, s>>>(g, f, a); break;
    case 3: d_expand_kernel<3><<<grid3(a), kBX, 0, s>>>(g, f, a); break;
    case 4: d_expand_kernel<4><<<grid3(a), kBX, 0, s>>>(g, f, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// intermediates (4 or 8 floats of (phi_k, rho), 6 of T, 19 f_i and 3P normal
// components per node), rounded up to 64 floats so that the FP64 staging
// behind them is aligned
size_t work_floats3(int N, size_t NN) {
  return (((N <= 3 ? 4 : 8) + 6 + Q3 + static_cast<size_t>(3) * N * (N - 1) / 2) * NN + 63) / 64 * 64;
}

// stored (post-collision, at the producing node) <-> post-streaming
// populations, all 19N planes of one node per thread
__global__ void __launch_bounds__(kBX) d_set_kernel(const double* __restrict__ fpost, float* __restrict__ f, DArgs a,
                                                    int planes) {
  Node p;
  if (!node_of(a, &p)) return;
  for (int pl = 0; pl < planes; ++pl) {
    const int i = pl % Q3;
    // stored(x) = post-streaming(x + e_i)
    f[static_cast<size_t>(pl) * p.NN + p.n] =
        static_cast<float>(fpost[static_cast<size_t>(pl) * p.NN + at(a, p, cx(i), cy(i), cz(i))]);
  }
}

// rest equilibrium per colour from the densities, in the stored form:
// stored(x) = post-streaming(x + e_i) = w_i rho_k(x + e_i)
__global__ void __launch_bounds__(kBX) d_init_kernel(const double* __restrict__ rho, float* __restrict__ f, DArgs a,
                                                     int nfluids) {
  Node p;
  if (!node_of(a, &p)) return;
  for (int k = 0; k < nfluids; ++k)
#pragma unroll
    for (int i = 0; i < Q3; ++i)
      f[(static_cast<size_t>(k) * Q3 + i) * p.NN + p.n] =
          static_cast<float>(w3d(i) * rho[static_cast<size_t>(k) * p.NN + at(a, p, cx(i), cy(i), cz(i))]);
}

__global__ void __launch_bounds__(kBX) d_get_kernel(const float* __restrict__ f, double* __restrict__ fpost, DArgs a,
                                                    int planes) {
  Node p;
  if (!node_of(a, &p)) return;
  for (int pl = 0; pl < planes; ++pl) {
    const int i = pl % Q3;
    fpost[static_cast<size_t>(pl) * p.NN + p.n] =
        static_cast<double>(f[static_cast<size_t>(pl) * p.NN + at(a, p, -cx(i), -cy(i), -cz(i))]);
  }
}

// FP64 per-plane sums: block (b, plane) sums a fixed stride-class of the
// plane in a fixed-order tree; the host adds the kSumBlocks partials of a
// plane in order, so the result does not depend on scheduling
constexpr int kSumBlocks = 64;
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) d_plane_sum_kernel(const float* __restrict__ f, size_t NN,
                                                                  double* __restrict__ out) {
  const int pl = blockIdx.y;
  double s = 0.0;
  for (size_t n = static_cast<size_t>(blockIdx.x) * kSumThreads + threadIdx.x; n < NN;
       n += static_cast<size_t>(kSumBlocks) * kSumThreads)
    s += static_cast<double>(f[static_cast<size_t>(pl) * NN + n]);
  __shared__ double sh[kSumThreads];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kSumThreads / 2; o > 0; o >>= 1) {
    if (static_cast<int>(threadIdx.x) < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[static_cast<size_t>(pl) * kSumBlocks + blockIdx.x] = sh[0];
}

double g_of3(double X) {  // Eq. 20
  if (X < -1.0) return 1.0;
  if (X < 0.0) return 1.0 - std::sqrt(1.0 - X * X);
  if (X <= 1.0) return std::sqrt(1.0 - X * X) - 1.0;
  return -1.0;
}

}  // namespace
}  // namespace lbm3

struct lbm3d_ctx {
  int N = 0, nx = 0, ny = 0, nz = 0;
  cudaStream_t stream = nullptr;
  float* buf[2] = {nullptr, nullptr};
  float* work = nullptr;
  double* sums = nullptr;
  int cur = 0;
  bool state_set = false;
  bool reduced = false;  // the storage form of the steps (LBM3_REDUCED)
  bool red = false;      // buf[cur] holds the reduced state (else populations)
  lbm3::DArgs args{};
  std::string msg;
};

namespace {

lbm3_status dfail(lbm3d_ctx* c, lbm3_status st, const std::string& m) {
  if (c) c->msg = m;
  return st;
}

lbm3_status dcuda(lbm3d_ctx* c, cudaError_t e, const char* where) {
  return dfail(c, LBM3_ECUDA, std::string("lbm3d: ") + where + ": " + cudaGetErrorString(e));
}

size_t nodes(const lbm3d_ctx* c) { return static_cast<size_t>(c->nx) * c->ny * c->nz; }

// the current state as stored populations: buf[cur] itself, or the reduced
// state expanded into the idle buffer
const float* stored_populations(lbm3d_ctx* c, cudaError_t* e) {
  *e = cudaSuccess;
  if (!c->red) return c->buf[c->cur];
  *e = lbm3::d_expand_any(c->N, c->buf[c->cur], c->buf[c->cur ^ 1], c->args, c->stream);
  return c->buf[c->cur ^ 1];
}

}  // namespace

extern "C" {

lbm3_status lbm3d_create(const lbm3d_params* p, void* cuda_stream, lbm3d_ctx** out) {
  if (!out) return LBM3_EINVAL;
  *out = nullptr;
  if (!p || !p->tau || !p->rho0 || !p->sigma) return LBM3_EINVAL;
  const int N = p->nfluids;
  if (N < 2 || N > lbm3::kMaxFluids3 || p->nx < 1 || p->ny < 1 || p->nz < 1 || p->ny > 65535 || p->nz > 65535)
    return LBM3_EINVAL;
  if (static_cast<double>(p->nx) * p->ny * p->nz * lbm3::Q3 * N >= 4294967296.0) return LBM3_EINVAL;
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
  lbm3d_ctx* c = new (std::nothrow) lbm3d_ctx();
  if (!c) return LBM3_ENOMEM;
  c->N = N;
  c->nx = p->nx;
  c->ny = p->ny;
  c->nz = p->nz;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->reduced = p->storage == LBM3_REDUCED;
  lbm3::DArgs& a = c->args;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  for (int k = 0; k < N; ++k) a.inv_nu[k] = static_cast<float>(3.0 / (p->tau[k] - 0.5));
  for (int k = 0; k < N; ++k)
    for (int l = k + 1; l < N; ++l) {
      const int q = lbm3::pair3(k, l, N);
      a.sigma[q] = static_cast<float>(p->sigma[k * N + l]);
      a.cpair[q] = static_cast<float>(1e6 / (p->rho0[k] * p->rho0[l]));
      for (int m = 0; m < N; ++m) {
        double gv = 0.0;
        if (m != k && m != l) {
          const double smk = p->sigma[m * N + k], sml = p->sigma[m * N + l], skl = p->sigma[k * N + l];
          gv = lbm3::g_of3((smk * smk + sml * sml - skl * skl) / (2.0 * smk * sml));  // Eqs. 18, 20
        }
        a.gjunc[q][m] = static_cast<float>(gv);
      }
    }
  a.beta0 = static_cast<float>(p->beta0);
  a.beta_A = p->beta_form == 0 ? 35.0f : 0.0f;
  for (int i = 0; i < lbm3::Q3; ++i) {
    const double len =
        std::sqrt(static_cast<double>(lbm3::cx(i) * lbm3::cx(i) + lbm3::cy(i) * lbm3::cy(i) + lbm3::cz(i) * lbm3::cz(i)));
    a.wrec[i] = static_cast<float>((p->recolor_form == 0 && i != 0) ? lbm3::w3d(i) / len : lbm3::w3d(i));
  }
  a.ndelta = static_cast<float>(p->normal_delta);
  const size_t NN = nodes(c);
  const size_t pop = static_cast<size_t>(lbm3::Q3) * N * NN * sizeof(float);
  void *b0 = nullptr, *b1 = nullptr, *w = nullptr, *sm = nullptr;
  if (cudaMalloc(&b0, pop) != cudaSuccess || cudaMalloc(&b1, pop) != cudaSuccess ||
      cudaMalloc(&w, lbm3::work_floats3(N, NN) * sizeof(float) + lbm3::Q3 * N * NN * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sm, static_cast<size_t>(lbm3::Q3) * N * lbm3::kSumBlocks * sizeof(double)) != cudaSuccess) {
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

lbm3_status lbm3d_set_populations(lbm3d_ctx* c, const double* f, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!f) return dfail(c, LBM3_EINVAL, "lbm3d_set_populations: NULL f");
  const size_t NN = nodes(c);
  const int planes = lbm3::Q3 * c->N;
  const double* src = f;
  // FP64 staging behind the intermediates in the work allocation
  double* staging = reinterpret_cast<double*>(c->work + lbm3::work_floats3(c->N, NN));
  if (!on_device) {
    cudaError_t e = cudaMemcpyAsync(staging, f, planes * NN * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return dcuda(c, e, "copy to the device");
    src = staging;
  }
  lbm3::d_set_kernel<<<lbm3::grid3(c->args), lbm3::kBX, 0, c->stream>>>(src, c->buf[c->cur], c->args, planes);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return dcuda(c, e, "lbm3d_set_populations");
  c->state_set = true;
  c->red = false;
  return LBM3_OK;
}

lbm3_status lbm3d_init(lbm3d_ctx* c, const double* rho, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!rho || on_device) return dfail(c, LBM3_EINVAL, "lbm3d_init: host densities rho[N][nz][ny][nx] required");
  const size_t NN = nodes(c);
  for (size_t n = 0; n < static_cast<size_t>(c->N) * NN; ++n)
    if (!(rho[n] >= 0.0)) return dfail(c, LBM3_EINVAL, "lbm3d_init: rho_k must be >= 0");
  // the densities go through the FP64 staging area (N of its 19 N planes)
  double* staging = reinterpret_cast<double*>(c->work + lbm3::work_floats3(c->N, NN));
  cudaError_t e = cudaMemcpyAsync(staging, rho, static_cast<size_t>(c->N) * NN * sizeof(double),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    lbm3::d_init_kernel<<<lbm3::grid3(c->args), lbm3::kBX, 0, c->stream>>>(staging, c->buf[c->cur], c->args, c->N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return dcuda(c, e, "lbm3d_init");
  c->state_set = true;
  c->red = false;
  return LBM3_OK;
}

lbm3_status lbm3d_step(lbm3d_ctx* c, int64_t n) {
  if (!c) return LBM3_EINVAL;
  if (n < 0) return dfail(c, LBM3_EINVAL, "lbm3d_step: n < 0");
  if (!c->state_set) return dfail(c, LBM3_ESTATE, "lbm3d_step: state not set");
  for (int64_t s = 0; s < n; ++s) {
    const cudaError_t e = lbm3::d_step_any(c->N, c->buf[c->cur], c->buf[c->cur ^ 1], c->work, c->args, c->stream,
                                           c->red, c->reduced);
    if (e != cudaSuccess) return dcuda(c, e, "lbm3d_step");
    c->cur ^= 1;
    c->red = c->reduced;
  }
  return LBM3_OK;
}

lbm3_status lbm3d_populations(lbm3d_ctx* c, double* f, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!f) return dfail(c, LBM3_EINVAL, "lbm3d_populations: NULL f");
  if (!c->state_set) return dfail(c, LBM3_ESTATE, "lbm3d_populations: state not set");
  const size_t NN = nodes(c);
  const int planes = lbm3::Q3 * c->N;
  double* dst = on_device ? f : reinterpret_cast<double*>(c->work + lbm3::work_floats3(c->N, NN));
  cudaError_t e;
  const float* src = stored_populations(c, &e);
  if (e == cudaSuccess) {
    lbm3::d_get_kernel<<<lbm3::grid3(c->args), lbm3::kBX, 0, c->stream>>>(src, dst, c->args, planes);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(f, dst, planes * NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return dcuda(c, e, "lbm3d_populations");
  return LBM3_OK;
}

lbm3_status lbm3d_fields(lbm3d_ctx* c, double* rho, double* u, double* p, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!c->state_set) return dfail(c, LBM3_ESTATE, "lbm3d_fields: state not set");
  const size_t NN = nodes(c);
  // the FP64 staging area holds the host case's outputs: N + 3 + 1 of its 19 N planes
  double* staging = reinterpret_cast<double*>(c->work + lbm3::work_floats3(c->N, NN));
  double* d_rho = rho ? (on_device ? rho : staging) : nullptr;
  double* d_u = u ? (on_device ? u : staging + static_cast<size_t>(c->N) * NN) : nullptr;
  double* d_p = p ? (on_device ? p : staging + static_cast<size_t>(c->N + 3) * NN) : nullptr;
  cudaError_t e = lbm3::d_fields_any(c->N, c->red, c->buf[c->cur], c->work, d_rho, d_u, d_p, c->args, c->stream);
  if (e == cudaSuccess && !on_device) {
    if (rho)
      e = cudaMemcpyAsync(rho, d_rho, static_cast<size_t>(c->N) * NN * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess && u)
      e = cudaMemcpyAsync(u, d_u, 3 * NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, d_p, NN * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return dcuda(c, e, "lbm3d_fields");
  return LBM3_OK;
}

lbm3_status lbm3d_mass(lbm3d_ctx* c, double* mass, double* mom) {
  if (!c) return LBM3_EINVAL;
  if (!c->state_set) return dfail(c, LBM3_ESTATE, "lbm3d_mass: state not set");
  const int planes = lbm3::Q3 * c->N;
  cudaError_t e;
  const float* src = stored_populations(c, &e);
  if (e == cudaSuccess) {
    lbm3::d_plane_sum_kernel<<<dim3(lbm3::kSumBlocks, planes), lbm3::kSumThreads, 0, c->stream>>>(src, nodes(c),
                                                                                                   c->sums);
    e = cudaGetLastError();
  }
  std::vector<double> h(static_cast<size_t>(planes) * lbm3::kSumBlocks);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), c->sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return dcuda(c, e, "lbm3d_mass");
  double mo[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < c->N; ++k) {
    double m = 0.0;
    for (int i = 0; i < lbm3::Q3; ++i) {
      double v = 0.0;
      for (int b = 0; b < lbm3::kSumBlocks; ++b) v += h[(static_cast<size_t>(k) * lbm3::Q3 + i) * lbm3::kSumBlocks + b];
      m += v;
      mo[0] += lbm3::cx(i) * v;
      mo[1] += lbm3::cy(i) * v;
      mo[2] += lbm3::cz(i) * v;
    }
    if (mass) mass[k] = m;
  }
  if (mom)
    for (int d = 0; d < 3; ++d) mom[d] = mo[d];
  return LBM3_OK;
}

lbm3_status lbm3d_destroy(lbm3d_ctx* c) {
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

const char* lbm3d_last_error(const lbm3d_ctx* c) { return c ? c->msg.c_str() : "lbm3d: NULL context"; }

}  // extern "C"
