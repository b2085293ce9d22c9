// Fused D2Q9 ternary colour-gradient step for sm_103a (arXiv 1808.08555, Sec. 2).
//
// One kernel does the whole time step for a strip of up to kTX columns and a
// run of H rows:
//   D stage  (row r+2): pulled populations -> rho_k, rho, phi_k = rho_k/rho
//                       (Eq. 30 read as a pull; rho_k after Eq. 30)
//   T stage  (row r+1): grad phi_k (Eq. fd1) -> G_kl, C_kl (Eq. 15),
//                       normals n_kl (regularised where G_kl -> 0), tension tensor
//                       T = sum_{k<l} sigma_kl C_kl |G_kl| (I - n_kl n_kl)
//                       (Eq. 11's double sum with the 1/2 folded into k<l)
//   C stage  (row r)  : F_s = div T (Eq. fd1 again), u (Eq. uk1), tau_f
//                       (Eqs. vis_1, tau), BGK + Guo (Eqs. 1-3, 5), beta_kl
//                       (Eqs. 18-20 or the alternatives), recolouring (Eq. 6),
//                       store f^ddagger at x (streaming happens in the next
//                       step's pull).
// Population rows reach shared memory by bulk asynchronous copies
// (cp.async.bulk + mbarrier complete_tx) issued by one producer warp into a
// ring of kSlots rows; four consumer warps run the three stages on rows
// r+2, r+1, r in lock step (two named barriers per row).  HBM traffic is one
// read and one write of the 27 populations per node; halo re-reads of
// neighbouring strips' columns are served by L2.
//
// Every mbarrier wait is bounded in time (kWaitNs).  A wait that gives up
// sets bit 0 of *err and marks the CTA aborted: the producer stops issuing
// copies, the consumers skip their arithmetic but keep every barrier, and the
// producer waits (bounded) for every copy it issued before the CTA exits.

#include <cstdint>

#include "lbm3_internal.h"

namespace lbm3 {
namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait
// n_kl = G_kl / |G_kl| is undefined where G_kl = 0 and makes the recolouring
// of Eq. 6 jump there; the normal is regularised as G / max(|G|, 0.1 phi_k
// phi_l).  Across a k-l interface |G_kl| is about 1.26 phi_k phi_l (tanh
// profile of Eq. 21), so the regularisation only acts near zeros of G_kl.
constexpr float kNormalDelta = 1e-1f;

struct Smem {
  float pop[kSlots][27][kPW];  // pulled-row ring, plane = k*9 + i
  float phi[4][4][kDW];        // phi_1, phi_2, phi_3, rho on 4 rows
  float T[3][3][kTW];          // T_xx, T_xy, T_yy on 3 rows
  float nrm[2][6][kTX];        // n_12, n_13, n_23 (x, y) on 2 rows
  unsigned long long full[kSlots];
  unsigned long long empty[kSlots];
  int abort_flag;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  [[maybe_unused]] unsigned long long state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(su32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  [[maybe_unused]] unsigned long long state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase with the given parity.  Returns false (after
// flagging the error and the CTA abort) if it did not complete in kWaitNs or
// another thread of the CTA already aborted.
__device__ bool mbar_wait(unsigned long long* bar, uint32_t parity, volatile int* abort_flag,
                          unsigned int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > kWaitNs) {
        *abort_flag = 1;
        atomicOr(err, 1u);
        return false;
      }
    }
  }
}

// Drain variant used on the abort path: waits (bounded) without consulting
// the abort flag, so that copies in flight land before the CTA exits.
__device__ void mbar_wait_drain(unsigned long long* bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > kWaitNs) return;
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory"); }

__device__ __forceinline__ int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Isotropic stencil of Eq. fd1 (1/c_s^2 = 3 folded in) at window column c of
// three rows (m = y-1, z = y, p = y+1).
__device__ __forceinline__ float ddx(const float* m, const float* z, const float* p, int c) {
  return (1.0f / 3.0f) * (z[c + 1] - z[c - 1]) + (1.0f / 12.0f) * ((p[c + 1] - p[c - 1]) + (m[c + 1] - m[c - 1]));
}
__device__ __forceinline__ float ddy(const float* m, const float* z, const float* p, int c) {
  return (1.0f / 3.0f) * (p[c] - m[c]) + (1.0f / 12.0f) * ((p[c + 1] + p[c - 1]) - (m[c + 1] + m[c - 1]));
}

// ----------------------------------------------------------------- producer
__device__ void produce(Smem& s, const StepArgs& a, int x0, int w, int y0, int nq, int lane) {
  const int nx = a.nx, ny = a.ny;
  const size_t N = static_cast<size_t>(nx) * ny;
  const uint32_t row_bytes = 27u * static_cast<uint32_t>(w + 8) * 4u;
  volatile int* abort_flag = &s.abort_flag;
  int issued = 0;
  for (int q = 0; q < nq; ++q) {
    const int slot = q % kSlots;
    // lane 0 decides for the whole warp, so the warp never diverges around
    // the __syncwarp() calls below
    int ok = 1;
    if (lane == 0) {
      if (q >= kSlots)
        ok = mbar_wait(&s.empty[slot], static_cast<uint32_t>((q / kSlots - 1) & 1), abort_flag, a.err) ? 1 : 0;
      if (ok && *abort_flag) ok = 0;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) break;
    if (lane == 0) mbar_arrive_expect_tx(&s.full[slot], row_bytes);
    __syncwarp();
    if (lane < 27) {
      const int i = lane % 9;
      const int src_row = wrap(y0 - 2 + q - ey(i), ny);
      const float* plane = a.fin + static_cast<size_t>(lane) * N + static_cast<size_t>(src_row) * nx;
      float* dst = &s.pop[slot][lane][0];
      // window [x0-4, x0+w+4) wrapped into [0, nx) in pieces; every piece
      // starts and ends on a multiple of 4 floats (nx % 4 == 0, x0 % 4 == 0)
      int start = x0 - 4, left = w + 8, off = 0;
      while (left > 0) {
        const int gx = wrap(start, nx);
        const int len = min(left, nx - gx);
        bulk_g2s(dst + off, plane + gx, static_cast<uint32_t>(len) * 4u, &s.full[slot]);
        start += len;
        off += len;
        left -= len;
      }
    }
    __syncwarp();
    issued = q + 1;
  }
  // Wait (bounded) until every issued row has landed, so that no copy can
  // target this CTA's shared memory after it exits.  On the normal path the
  // consumers wait for the same phases, so this costs nothing.
  for (int q = (issued > kSlots ? issued - kSlots : 0); q < issued; ++q)
    mbar_wait_drain(&s.full[q % kSlots], static_cast<uint32_t>((q / kSlots) & 1));
}

// ---------------------------------------------------------------- consumers
template <int MODE>
__device__ void consume(Smem& s, const StepArgs& a, int x0, int w, int y0, int nq, int tid) {
  const int nx = a.nx;
  const size_t N = static_cast<size_t>(nx) * a.ny;
  volatile int* abort_flag = &s.abort_flag;
  bool dead = false;

  for (int q = 0; q < nq; ++q) {
    // ---------------- D stage: densities on row y0-2+q, columns x0-2 .. x0+w+1
    const int ps = q % kSlots;
    if (!dead) dead = !mbar_wait(&s.full[ps], static_cast<uint32_t>((q / kSlots) & 1), abort_flag, a.err);
    if (!dead) {
      float(*pp)[kPW] = s.pop[ps];
      float(*ph)[kDW] = s.phi[q & 3];
      for (int c = tid; c < w + 4; c += kConsumers) {
        float rk[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float acc = 0.0f;
#pragma unroll
          for (int i = 0; i < 9; ++i) acc += pp[k * 9 + i][c + 2 - ex(i)];
          rk[k] = acc;
        }
        const float rho = rk[0] + rk[1] + rk[2];
        const float ir = 1.0f / rho;
        ph[0][c] = rk[0] * ir;
        ph[1][c] = rk[1] * ir;
        ph[2][c] = rk[2] * ir;
        ph[3][c] = rho;
      }
    }
    consumers_sync();

    // ---------------- T stage: tension tensor on row y0-3+q, columns x0-1 .. x0+w
    if (q >= 2 && !dead) {
      const float(*pm)[kDW] = s.phi[(q - 2) & 3];
      const float(*pz)[kDW] = s.phi[(q - 1) & 3];
      const float(*pq)[kDW] = s.phi[q & 3];
      float(*Tt)[kTW] = s.T[q % 3];
      float(*nn)[kTX] = s.nrm[q & 1];
      for (int c = tid; c < w + 2; c += kConsumers) {
        const int cc = c + 1;  // phi window column of this node
        float ph[3], gx[3], gy[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          ph[k] = pz[k][cc];
          gx[k] = ddx(pm[k], pz[k], pq[k], cc);
          gy[k] = ddy(pm[k], pz[k], pq[k], cc);
        }
        const float rho = pz[3][cc];
        float txx = 0.0f, txy = 0.0f, tyy = 0.0f;
        float nv[6];
#pragma unroll
        for (int q2 = 0; q2 < 3; ++q2) {
          const int k = q2 < 2 ? 0 : 1;
          const int l = q2 == 0 ? 1 : 2;
          // G_kl = phi_l grad phi_k - phi_k grad phi_l
          const float Gx = ph[l] * gx[k] - ph[k] * gx[l];
          const float Gy = ph[l] * gy[k] - ph[k] * gy[l];
          const float g2 = Gx * Gx + Gy * Gy;
          const float mag = sqrtf(g2);
          if (g2 > 1e-30f) {
            const float ck = fminf(a.cpair[q2] * (ph[k] * rho) * (ph[l] * rho), 1.0f);
            // sigma C |G| (I - n n) = sigma C (|G|^2 I - G G) / |G|
            const float sc = a.sigma[q2] * ck / mag;
            txx += sc * Gy * Gy;
            txy -= sc * Gx * Gy;
            tyy += sc * Gx * Gx;
          }
          // recolouring normal G / max(|G|, kNormalDelta phi_k phi_l): the unit
          // normal wherever a k-l interface exists, continuous to 0 where G -> 0
          const float den = fmaxf(mag, kNormalDelta * ph[k] * ph[l]);
          const float rden = den > 1e-30f ? 1.0f / den : 0.0f;  // |n| <= 1; tiny den -> 0
          nv[2 * q2] = Gx * rden;
          nv[2 * q2 + 1] = Gy * rden;
        }
        Tt[0][c] = txx;
        Tt[1][c] = txy;
        Tt[2][c] = tyy;
        if (c >= 1 && c <= w) {
#pragma unroll
          for (int j = 0; j < 6; ++j) nn[j][c - 1] = nv[j];
        }
      }
    }
    consumers_sync();

    // ---------------- C stage: row y0-4+q, columns x0 .. x0+w-1
    if (q >= 4 && !dead && tid < w) {
      const int row = y0 - 4 + q;
      float(*pp)[kPW] = s.pop[(q - 2) % kSlots];
      const float(*Tm)[kTW] = s.T[(q - 2) % 3];
      const float(*Tz)[kTW] = s.T[(q - 1) % 3];
      const float(*Tp)[kTW] = s.T[q % 3];
      const float(*nn)[kTX] = s.nrm[(q - 1) & 1];
      const int c = tid;
      float f[27];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 9; ++i) f[k * 9 + i] = pp[k * 9 + i][c + 4 - ex(i)];
      float rk[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) acc += f[k * 9 + i];
        rk[k] = acc;
      }
      const float rho = rk[0] + rk[1] + rk[2];
      const float ir = 1.0f / rho;
      // F_s = div T (Eq. 11), T window column of this node is c + 1
      const int tc = c + 1;
      const float Fx = ddx(Tm[0], Tz[0], Tp[0], tc) + ddy(Tm[1], Tz[1], Tp[1], tc);
      const float Fy = ddx(Tm[1], Tz[1], Tp[1], tc) + ddy(Tm[2], Tz[2], Tp[2], tc);
      float fi[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) fi[i] = f[i] + f[9 + i] + f[18 + i];
      const float mx = (fi[1] - fi[3]) + (fi[5] - fi[6]) + (fi[8] - fi[7]);
      const float my = (fi[2] - fi[4]) + (fi[5] - fi[8]) + (fi[6] - fi[7]);
      // Eq. uk1
      const float ux = (mx + 0.5f * Fx) * ir;
      const float uy = (my + 0.5f * Fy) * ir;
      if (MODE == MODE_FIELDS) {
        const size_t idx = static_cast<size_t>(row) * nx + (x0 + c);
        if (a.out_rho) {
          a.out_rho[idx] = rk[0];
          a.out_rho[N + idx] = rk[1];
          a.out_rho[2 * N + idx] = rk[2];
        }
        if (a.out_ux) a.out_ux[idx] = ux;
        if (a.out_uy) a.out_uy[idx] = uy;
        if (a.out_p) a.out_p[idx] = static_cast<double>(rho) / 3.0;
      } else {
        // Eqs. vis_1 / tau: rho/nu = sum rho_k/nu_k, tau_f = 3 nu + 1/2
        const float snu = rk[0] * a.inv_nu[0] + rk[1] * a.inv_nu[1] + rk[2] * a.inv_nu[2];
        const float tauf = 3.0f * (rho / snu) + 0.5f;
        const float om = 1.0f / tauf;
        const float uu = ux * ux + uy * uy;
        const float uF = ux * Fx + uy * Fy;
        const float gpre = 1.0f - 0.5f * om;
        float fd[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const float eu = ex(i) * ux + ey(i) * uy;
          const float eF = ex(i) * Fx + ey(i) * Fy;
          const float feq = wt(i) * rho * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
          const float guo = wt(i) * gpre * (3.0f * (eF - uF) + 9.0f * eu * eF);
          fd[i] = fi[i] - om * (fi[i] - feq) + guo;  // Eqs. 1, 2, 5
        }
        // segregation parameters beta_kl (pairs 12, 13, 23)
        const float prod = rk[0] * rk[1] * rk[2] * (ir * ir * ir);
        const float cb = fminf(a.beta_A * prod, 1.0f);
        float Rx[3], Ry[3];
#pragma unroll
        for (int q2 = 0; q2 < 3; ++q2) {
          const int k = q2 < 2 ? 0 : 1;
          const int l = q2 == 0 ? 1 : 2;
          const float b = a.beta0 * (1.0f + cb * a.beta_h[q2]);
          const float amp = b * rk[k] * rk[l] * ir;
          Rx[q2] = amp * nn[2 * q2][c];
          Ry[q2] = amp * nn[2 * q2 + 1][c];
        }
        // sum_{l != k} beta_kl (rho_k rho_l / rho) n_kl, with n_lk = -n_kl
        const float Vx[3] = {Rx[0] + Rx[1], Rx[2] - Rx[0], -Rx[1] - Rx[2]};
        const float Vy[3] = {Ry[0] + Ry[1], Ry[2] - Ry[0], -Ry[1] - Ry[2]};
        const size_t base = static_cast<size_t>(row) * nx + (x0 + c);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float phk = rk[k] * ir;
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            const float en = ex(i) * Vx[k] + ey(i) * Vy[k];
            a.fout[static_cast<size_t>(k * 9 + i) * N + base] = phk * fd[i] + a.wrec[i] * en;  // Eq. 6
          }
        }
      }
    }
    // release the population row that the C stage (or, for the first two
    // halo rows, the D stage) finished with
    if (q >= 2) mbar_arrive(&s.empty[(q - 2) % kSlots]);
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) fused_step_kernel(StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  const int strip = blockIdx.x % a.nstrips;
  const int chunk = blockIdx.x / a.nstrips;
  const int x0 = strip * kTX;
  const int w = min(kTX, a.nx - x0);
  const int y0 = chunk * a.rows_per_cta;
  const int h = min(a.rows_per_cta, a.ny - y0);
  if (w <= 0 || h <= 0) return;
  const int nq = h + 4;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int j = 0; j < kSlots; ++j) {
      mbar_init(&s.full[j], 1);
      mbar_init(&s.empty[j], kConsumers);
    }
    s.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid >= kConsumers) {
    produce(s, a, x0, w, y0, nq, tid - kConsumers);
  } else {
    consume<MODE>(s, a, x0, w, y0, nq, tid);
  }
}

}  // namespace

size_t step_smem_bytes() { return sizeof(Smem); }

cudaError_t step_configure() {
  cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<MODE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sizeof(Smem)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fused_step_kernel<MODE_FIELDS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(sizeof(Smem)));
}

int step_occupancy(int* blocks_per_sm) {
  return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, fused_step_kernel<MODE_STEP>, kThreads, sizeof(Smem)));
}

cudaError_t launch_step(const StepArgs& a, int grid, int mode, cudaStream_t st) {
  if (mode == MODE_STEP)
    fused_step_kernel<MODE_STEP><<<grid, kThreads, sizeof(Smem), st>>>(a);
  else
    fused_step_kernel<MODE_FIELDS><<<grid, kThreads, sizeof(Smem), st>>>(a);
  return cudaGetLastError();
}

}  // namespace lbm3
