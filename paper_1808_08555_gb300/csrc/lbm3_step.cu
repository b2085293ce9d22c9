// Fused D2Q9 ternary colour-gradient step for sm_103a (arXiv 1808.08555, Sec. 2).
//
// One kernel does the whole time step for a strip of up to kTX columns and a
// run of H rows.  Rows are indexed q = 0 .. H+3 from y0-2; each iteration j
// of the march handles two rows in each of three stages:
//   D stage  (rows 2j, 2j+1):   pulled populations -> rho_k, rho and
//                               phi_k = rho_k/rho (Eq. 30 read as a pull;
//                               rho_k as after Eq. 30)
//   T stage  (rows 2j-1, 2j):   grad phi_k (Eq. fd1) -> G_kl, C_kl (Eq. 15),
//                               normals n_kl (optionally regularised where
//                               G_kl -> 0) and
//                               the tension tensor
//                               T = sum_{k<l} sigma_kl C_kl |G_kl| (I - n n)
//                               (Eq. 11's double sum, 1/2 folded into k<l)
//   C stage  (rows 2j-2, 2j-1): F_s = div T (Eq. fd1 again), u (Eq. uk1),
//                               tau_f (Eqs. vis_1, tau), BGK + Guo (Eqs. 1-3,
//                               5), beta_kl (Eqs. 18-20 or the alternatives),
//                               recolouring (Eq. 6); store f^ddagger at x
//                               (streaming happens in the next step's pull).
// Population rows reach shared memory by 3D tiled TMA loads
// (cp.async.bulk.tensor + mbarrier complete_tx): per row three boxes of
// 9 planes x 132 columns, issued by one producer warp into a ring of kSlots
// rows; eight consumer warps run the stages in lock step (two named barriers
// per pair of rows).  Only the D stage reads a population row: it also
// leaves the node's total distribution f_i = sum_k f_{i,k} in a ring of its
// own for the C stage, so each population row is released as soon as its D
// stage is done and the loads run almost two iterations ahead.  The stages
// hand each other one vector per node and quantity (phi and rho, f_i, the
// tension tensor, the normals), and the arithmetic runs on packed FP32 pairs
// (directions e and -e, x and y).  HBM traffic is one read and one write of
// the 27 populations per node; halo re-reads of neighbouring strips' columns
// are served by L2.
//
// Reduced state (ST_RED): the ring holds source rows of the reduced state
// (phi_k, f^dagger_i, V_k per node; see lbm3_internal.h), two TMA boxes per
// row into six slots; the D stage rebuilds each pulled population from its
// source node with the C stage's own FP32 operations (red_pop), so the
// reduced form's trajectory is the FP32 form's, bit for bit, at 72 instead of
// 108 bytes per node and direction of the step.  The C stage stores 9 values
// per node (three float4 and six floats) instead of 27.
//
// Every mbarrier wait is bounded in time (kWaitNs).  A wait that gives up
// sets bit 0 of *err and marks the CTA aborted: the producer stops issuing
// copies, the consumers skip their arithmetic but keep every barrier, and the
// producer waits (bounded) for every copy it issued before the CTA exits.

#include <cstdint>
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm3_internal.h"

namespace lbm3 {
namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

struct Smem {
  // pulled-row ring (row q in slot q % kSlots): three TMA boxes of 9 planes x
  // kPW columns, one per direction group, each starting on a 128-byte boundary
  // (the reduced state uses the same bytes as kRedSlots slots of kRedSlotFloats)
  float pop[kSlots][3 * kGroupFloats];
  float4 phi[6][kDW];          // (phi_1, phi_2, phi_3, rho) of row q in slot q % 6
  float4 fi4[6][2][kTX];       // (f_1, f_2, f_3, f_4), (f_5, f_6, f_7, f_8) of row q in slot q % 6
  float fi0[6][kTX];           // f_0 of row q in slot q % 6
  float4 T[4][kTW];            // (T_xx, T_xy, T_xy, T_yy) of row q in slot q % 4: the pairs the divergence uses
  float4 nrm01[3][kTX];        // (x, y) of n_12 and n_13 of row q in slot q % 3
  float2 nrm2[3][kTX];         // (x, y) of n_23
  unsigned long long full[kMaxSlots];
  unsigned long long empty[kMaxSlots];
  int abort_flag;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Packed FP32 pairs (the f32x2 add / mul / fma of sm_100 and later): each
// lane is rounded exactly as the scalar operation, so a pair of identical
// scalar expressions is evaluated in one instruction.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// hardware reciprocal estimate (rcp.approx: at most 1 ulp off; rho is never
// denormal), one instruction
__device__ __forceinline__ float rcp_est(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
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
__device__ __noinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, volatile int* abort_flag,
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

// 3D tiled TMA load of one box (boxw, 1, 9) at (x, y, z) into shared memory,
// completing on the given mbarrier.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}

// 4D tiled TMA load of one box (16, boxw/4, 1, planes) at (0, x, y, 0): the
// float4 planes of the reduced state, four columns per innermost run.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(0), "r"(su32(bar))
      : "memory");
}

// Ring slot of the reduced state's source row r.
__device__ __forceinline__ float* red_slot(Smem& s, int r) {
  return &s.pop[0][0] + (r % kRedSlots) * kRedSlotFloats;
}

// Slots of the three source rows q, q + 1, q + 2 that march row q pulls from
// (one modulo instead of three).
struct RedRows {
  const float* row[3];
};
__device__ __forceinline__ RedRows red_rows(Smem& s, int q) {
  int j = q % kRedSlots;
  RedRows r;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    r.row[t] = &s.pop[0][0] + j * kRedSlotFloats;
    j = j + 1 == kRedSlots ? 0 : j + 1;
  }
  return r;
}

// Ring column of window column 0 (padded column x0) in the 16-bit deviation
// box of a slot; the FP32, rho' and reduced-state boxes start at x0 itself.
// (Every box starts at the strip's own window, the last strip's box running
// past the end of the row where it is narrower than the box: TMA fills those
// columns with zeros without reading memory, and no stage reads them.  A box
// shifted left to stay inside the row re-read up to kPW - w - 8 columns of
// the previous strip from DRAM for every row.)
struct RingCols {
  int d;
};
__device__ __forceinline__ RingCols ring_cols(int x0) {
  RingCols c;
  c.d = x0 & 7;
  return c;
}

// Pulled value of colour k, direction i at window column wc of one slot:
// read directly (FP32), or rebuilt as w_i rho'_k + d (16-bit deviations).
template <int ST>
__device__ __forceinline__ float popv(const float* slot, int k, int i, int wc, const RingCols& rc) {
  if (ST == ST_FP32) return slot[dir_group(i) * kGroupFloats + (3 * k + dir_pos(i)) * kPW + wc];
  const unsigned short* dv = reinterpret_cast<const unsigned short*>(slot);
  const float* rr = reinterpret_cast<const float*>(dv + 3 * kDevGroupHalfs);
  return fmaf(wt(i), rr[dir_group(i) * kRhoGroupFloats + k * kPW + wc],
              dec16<ST>(dv[dir_group(i) * kDevGroupHalfs + (3 * k + dir_pos(i)) * kDevBoxCols + wc + rc.d]));
}

__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory"); }

__device__ __forceinline__ int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// ----------------------------------------------------------------- producer
// Row q of the march (y = y0 - 2 + q) needs, for the directions with
// e_y = 1 - g, the source row y - e_y: three TMA boxes per row, one per group
// g, each bringing the 9 planes of that group over columns [tma_x, tma_x + boxw).
template <int ST, bool STALL>
__device__ void produce(Smem& s, const StepArgs& a, const CUtensorMap* map, const CUtensorMap* map1, int x0,
                        int y0, int nq, int lane) {
  constexpr int STI = st_in(ST);
  constexpr bool RED = STI == ST_RED;
  constexpr int NS = RED ? kRedSlots : kSlots;
  // the reduced state is loaded by source row (y0 - 3 + r, r = 0 .. nq + 1);
  // the other storages by march row (each row's three boxes from its three
  // source rows)
  const int nrows = RED ? nq + 2 : nq;
  const int ny = a.ny;
  const uint32_t row_bytes = STI == ST_FP32 ? 27u * kPW * 4u
                             : RED          ? (kRedVecPlanes * 4u + kRedSclPlanes) * kPW * 4u
                                            : 27u * kDevBoxCols * 2u + 9u * kPW * 4u;
  const int tma_x = x0;
  const int dev_x = x0 & ~7;
  volatile int* abort_flag = &s.abort_flag;
  int issued = 0;
  for (int q = 0; q < nrows; ++q) {
    const int slot = q % NS;
    // lane 0 decides for the whole warp, so the warp never diverges around
    // the __syncwarp() calls below
    int ok = 1;
    if (lane == 0) {
      if (q >= NS)
        ok = mbar_wait(&s.empty[slot], static_cast<uint32_t>((q / NS - 1) & 1), abort_flag, a.err) ? 1 : 0;
      if (ok && *abort_flag) ok = 0;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) break;
    if (lane == 0) mbar_arrive_expect_tx(&s.full[slot], row_bytes);
    __syncwarp();
    // testing hook (lbm3_debug_stall_row, a separate instantiation): the row
    // is announced but never copied, so the consumers' bounded waits run out
    const bool stall = STALL && q == a.stall_row && blockIdx.x == 0;
    if (stall) {
    } else if (RED) {
      const int src_row = wrap(y0 - 3 + q, ny);
      float* sl = red_slot(s, q);
      if (lane == 0)
        tma_load_4d(sl, map, tma_x / 4, src_row, &s.full[slot]);
      else if (lane == 1)
        tma_load_3d(sl + kRedVecFloats, map1, tma_x, src_row, 0, &s.full[slot]);
    } else if (STI == ST_FP32) {
      if (lane < 3) {
        const int g = lane;  // e_y = 1 - g
        const int src_row = wrap(y0 - 2 + q - (1 - g), ny);
        tma_load_3d(&s.pop[slot][g * kGroupFloats], map, tma_x, src_row, 9 * g, &s.full[slot]);
      }
    } else if (lane < 6) {
      const int g = lane % 3;  // e_y = 1 - g; lanes 0-2 deviations, 3-5 rho'
      const int src_row = wrap(y0 - 2 + q - (1 - g), ny);
      unsigned short* dv = reinterpret_cast<unsigned short*>(&s.pop[slot][0]);
      if (lane < 3)
        tma_load_3d(dv + g * kDevGroupHalfs, map, dev_x, src_row, 9 * g, &s.full[slot]);
      else
        tma_load_3d(reinterpret_cast<float*>(dv + 3 * kDevGroupHalfs) + g * kRhoGroupFloats, map1, tma_x, src_row, 0,
                    &s.full[slot]);
    }
    __syncwarp();
    issued = q + 1;
  }
  // Wait (bounded) until every issued row has landed, so that no copy can
  // target this CTA's shared memory after it exits.  On the normal path the
  // consumers wait for the same phases, so this costs nothing.
  for (int q = (issued > NS ? issued - NS : 0); q < issued; ++q)
    mbar_wait_drain(&s.full[q % NS], static_cast<uint32_t>((q / NS) & 1));
}

// ---------------------------------------------------------------- consumers
// phi_k = rho_k / rho in FP32 such that the three fractions sum to one and a
// single-fluid node gets exactly 1: the largest fraction is taken as the
// complement of the two others.  With plain products rho_k * (1/rho) a pure
// node gets 1 +- 1 ulp, always with the same sign for the same density, and
// the recolouring then creates or destroys that fluid's mass at a steady
// ~1e-8 relative per step.  The complement makes the sum exact whatever the
// rounding of 1/rho, so the hardware estimate serves.  Computed once per
// node (D stage) and read from the phi ring by the later stages.
__device__ __forceinline__ void colour_fractions(float r0, float r1, float r2, float* p, float* rho_out) {
  const float rho = (r0 + r1) + r2;
  const float ir = rcp_est(rho);
  float p0 = r0 * ir, p1 = r1 * ir, p2 = r2 * ir;
  if (r0 >= r1 && r0 >= r2) {
    p0 = (1.0f - p1) - p2;
  } else if (r1 >= r2) {
    p1 = (1.0f - p0) - p2;
  } else {
    p2 = (1.0f - p0) - p1;
  }
  p[0] = p0;
  p[1] = p1;
  p[2] = p2;
  *rho_out = rho;
}

// D stage, one node: row q (window slot), density column c in [0, w+4), i.e.
// x = x0 - 2 + c.  The pulled value of direction i sits at window column
// c + 2 - e_ix of row q's slot.  The 27 values are held as packed pairs of
// directions (1, 2), (3, 4), (5, 6), (7, 8) per colour: rho_k sums a colour's
// pairs, f_i = sum_k f_{i,k} sums the colours of a pair.  Nodes of the
// strip itself (c in [2, w+2)) leave f_i in the f ring for the C stage.
template <int ST>
__device__ __forceinline__ void stage_density(Smem& s, int q, int c, int w, const RingCols& rc) {
  const float* pp = s.pop[q % kSlots];
  const int wc = c + 2;
  float f0[3], r[3];
  float2 F[4];  // per pair of directions: sum over the colours so far
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    f0[k] = popv<ST>(pp, k, 0, wc, rc);
    float2 A;  // running sum of this colour's pairs
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = 2 * m + 1, j = 2 * m + 2;
      const float2 P = make_float2(popv<ST>(pp, k, i, wc - ex(i), rc), popv<ST>(pp, k, j, wc - ex(j), rc));
      A = m == 0 ? P : add2(A, P);
      F[m] = k == 0 ? P : add2(F[m], P);
    }
    r[k] = f0[k] + (A.x + A.y);
  }
  float phk[3], rho;
  colour_fractions(r[0], r[1], r[2], phk, &rho);
  const int fs = q % 6;
  s.phi[fs][c] = make_float4(phk[0], phk[1], phk[2], rho);
  if (c >= 2 && c < w + 2) {
#pragma unroll
    for (int m = 0; m < 2; ++m) s.fi4[fs][m][c - 2] = make_float4(F[2 * m].x, F[2 * m].y, F[2 * m + 1].x, F[2 * m + 1].y);
    s.fi0[fs][c - 2] = (f0[0] + f0[1]) + f0[2];
  }
}

// The three colours' pulled populations of direction I at the node of
// window column wc (reduced state): from the source node x - e_I, in source
// row q + 1 - e_Iy and window column wc - e_Ix, formed by red_pop.  (Packing
// colours 1 and 2 into FP32 pairs here spills registers at the 96-register
// cap of two CTAs per SM.)
template <int I>
__device__ __forceinline__ void pull_red(const RedRows& rr, const StepArgs& a, int wc, float* v) {
  const float* sl = rr.row[1 - ey(I)];
  const float4* vec = reinterpret_cast<const float4*>(sl);
  const int col = wc - ex(I);
  const float4 A = vec[col];  // (phi_1, phi_2, phi_3, fd_0)
  float4 X = make_float4(0.0f, 0.0f, 0.0f, 0.0f), Y = X;
  if (ex(I) != 0 || I == 1) X = vec[kPW + col];      // (V_1x, V_2x, V_3x, fd_1)
  if (ey(I) != 0 || I == 2) Y = vec[2 * kPW + col];  // (V_1y, V_2y, V_3y, fd_2)
  const float fd = I == 0 ? A.w : (I == 1 ? X.w : (I == 2 ? Y.w : sl[kRedVecFloats + (I - 3) * kPW + col]));
  v[0] = red_pop(I, A.x, fd, X.x, Y.x, a.wrec);
  v[1] = red_pop(I, A.y, fd, X.y, Y.y, a.wrec);
  v[2] = red_pop(I, A.z, fd, X.z, Y.z, a.wrec);
}

// D stage, one node, reduced state: the 27 pulled populations rebuilt from
// their source nodes, one direction at a time, summed as stage_density sums
// them (each lane of its packed pairs is the same scalar addition, in the
// same order), so every result equals the FP32 storage's.  Directions are
// taken one by one so that only one source node's values are live at a time.
__device__ __forceinline__ void stage_density_red(Smem& s, const StepArgs& a, int q, int c, int w) {
  const int wc = c + 2;
  const RedRows rr = red_rows(s, q);
  float f0[3], v[3];
  float Ax[3], Ay[3], Fx[4], Fy[4];  // lanes of the per-colour pair sums A and the pair totals F
  pull_red<0>(rr, a, wc, f0);
  auto take = [&](int lane, int m) {  // lane 0: direction 2m+1, lane 1: 2m+2
    float* Acc = lane == 0 ? Ax : Ay;
#pragma unroll
    for (int k = 0; k < 3; ++k) Acc[k] = m == 0 ? v[k] : Acc[k] + v[k];
    (lane == 0 ? Fx : Fy)[m] = (v[0] + v[1]) + v[2];
  };
  pull_red<1>(rr, a, wc, v);
  take(0, 0);
  pull_red<2>(rr, a, wc, v);
  take(1, 0);
  pull_red<3>(rr, a, wc, v);
  take(0, 1);
  pull_red<4>(rr, a, wc, v);
  take(1, 1);
  pull_red<5>(rr, a, wc, v);
  take(0, 2);
  pull_red<6>(rr, a, wc, v);
  take(1, 2);
  pull_red<7>(rr, a, wc, v);
  take(0, 3);
  pull_red<8>(rr, a, wc, v);
  take(1, 3);
  float r[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) r[k] = f0[k] + (Ax[k] + Ay[k]);
  float phk[3], rho;
  colour_fractions(r[0], r[1], r[2], phk, &rho);
  const int fs = q % 6;
  s.phi[fs][c] = make_float4(phk[0], phk[1], phk[2], rho);
  if (c >= 2 && c < w + 2) {
#pragma unroll
    for (int m = 0; m < 2; ++m) s.fi4[fs][m][c - 2] = make_float4(Fx[2 * m], Fy[2 * m], Fx[2 * m + 1], Fy[2 * m + 1]);
    s.fi0[fs][c - 2] = (f0[0] + f0[1]) + f0[2];
  }
}

// T stage, one node: row q, T-window column c in [0, w+2), x = x0 - 1 + c.
// FORCE 0 stores the tension tensor T of Eq. 11; FORCE 1 (the perturbation
// operator of Eqs. phi1 / phi_old) stores S = sum_kl (9/2) sigma_kl C_kl |G_kl|
// n_kl n_kl in the same three slots, from which Phi_i = (w_i e_i.S.e_i -
// B_i tr S) / tau_f at the node itself.
template <int FORCE>
__device__ __forceinline__ void stage_tension(Smem& s, const StepArgs& a, int q, int c, int w) {
  const float4* pm = s.phi[(q - 1) % 6];
  const float4* pz = s.phi[q % 6];
  const float4* pq = s.phi[(q + 1) % 6];
  const int cc = c + 1;  // phi-window column of this node
  // the nine (phi_1, phi_2, phi_3, rho) of the stencil, one vector load each;
  // the gradients run on the packed pairs (phi_1, phi_2) and (phi_3, rho)
  // (the rho lane is computed and dropped)
  const float4 C = pz[cc], W = pz[cc - 1], E = pz[cc + 1];
  const float4 SW = pm[cc - 1], S = pm[cc], SE = pm[cc + 1];
  const float4 NW = pq[cc - 1], Nn = pq[cc], NE = pq[cc + 1];
  auto lo = [](const float4& v) { return make_float2(v.x, v.y); };
  auto hi = [](const float4& v) { return make_float2(v.z, v.w); };
  // Eq. fd1 with 1/c_s^2 = 3: 3 (1/9) = 1/3 on the axes, 3 (1/36) = 1/12 on the diagonals
  const float2 c3 = bc2(1.0f / 3.0f), c12 = bc2(1.0f / 12.0f);
  const float2 gx01 = fma2(c12, add2(sub2(lo(NE), lo(NW)), sub2(lo(SE), lo(SW))), mul2(c3, sub2(lo(E), lo(W))));
  const float2 gy01 = fma2(c12, sub2(add2(lo(NE), lo(NW)), add2(lo(SE), lo(SW))), mul2(c3, sub2(lo(Nn), lo(S))));
  const float2 gx2r = fma2(c12, add2(sub2(hi(NE), hi(NW)), sub2(hi(SE), hi(SW))), mul2(c3, sub2(hi(E), hi(W))));
  const float2 gy2r = fma2(c12, sub2(add2(hi(NE), hi(NW)), add2(hi(SE), hi(SW))), mul2(c3, sub2(hi(Nn), hi(S))));
  const float ph[3] = {C.x, C.y, C.z};
  const float gx[3] = {gx01.x, gx01.y, gx2r.x};
  const float gy[3] = {gy01.x, gy01.y, gy2r.x};
  const float rho2 = C.w * C.w;
  float txx = 0.0f, txy = 0.0f, tyy = 0.0f;
  float2 nv[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int k = p < 2 ? 0 : 1;
    const int l = p == 0 ? 1 : 2;
    // G_kl = phi_l grad phi_k - phi_k grad phi_l
    const float2 G = fma2(bc2(ph[l]), make_float2(gx[k], gy[k]),
                          neg2(mul2(bc2(ph[k]), make_float2(gx[l], gy[l]))));
    const float Gx = G.x, Gy = G.y;
    const float g2 = Gx * Gx + Gy * Gy;
    const float pp = ph[k] * ph[l];
    float mag = 0.0f;
    if (g2 > 1e-30f) {
      // hardware estimate (<= 2 ulp): it scales the tension and the normal's
      // length, neither of which moves mass
      const float rinv = rsqrtf(g2);
      mag = g2 * rinv;
      const float ck = fminf(a.cpair[p] * pp * rho2, 1.0f);  // Eq. 15 with rho_k = phi_k rho
      if (FORCE == 0) {
        // sigma C |G| (I - n n) = sigma C (|G|^2 I - G G) / |G|
        const float sc = a.sigma[p] * ck * rinv;
        txx = fmaf(sc * Gy, Gy, txx);
        txy = fmaf(-sc * Gx, Gy, txy);
        tyy = fmaf(sc * Gx, Gx, tyy);
      } else {
        // (9/2) sigma C |G| n n = (9/2) sigma C G G / |G|
        const float sc = 4.5f * a.sigma[p] * ck * rinv;
        txx = fmaf(sc * Gx, Gx, txx);
        txy = fmaf(sc * Gx, Gy, txy);
        tyy = fmaf(sc * Gy, Gy, tyy);
      }
    }
    // recolouring normal G / max(|G|, delta phi_k phi_l): with delta = 0 the
    // unit normal G/|G| of Eq. 6; with delta > 0 the unit normal wherever
    // |G| >= delta phi_k phi_l (across a k-l interface |G| is about
    // 1.26 phi_k phi_l on the tanh profile of Eq. 21), going continuously to
    // 0 where G -> 0.  0 at or below the |G| cutoff of the tension (no k-l
    // interface).
    const float den = fmaxf(mag, a.ndelta * pp);
    const float rden = g2 > 1e-30f ? __fdividef(1.0f, den) : 0.0f;  // |n| <= 1
    nv[p] = mul2(G, bc2(rden));
  }
  s.T[q & 3][c] = make_float4(txx, txy, txy, tyy);
  if (c >= 1 && c <= w) {
    const int ns = q % 3;
    s.nrm01[ns][c - 1] = make_float4(nv[0].x, nv[0].y, nv[1].x, nv[1].y);
    s.nrm2[ns][c - 1] = nv[2];
  }
}

// C stage, one node: row q (output row y0 - 2 + q), column c in [0, w).
template <int MODE, int ST, int FORCE>
__device__ __forceinline__ void stage_collide(Smem& s, const StepArgs& a, int q, int c, int x0, int y0) {
  const float4* Tm = s.T[(q - 1) & 3];
  const float4* Tz = s.T[q & 3];
  const float4* Tp = s.T[(q + 1) & 3];
  // colour fractions and density from the D stage (the phi and f rings keep
  // six rows, so the next iteration's D stage writes other slots)
  const float4 pr = s.phi[q % 6][c + 2];
  const float phi0 = pr.x, phi1 = pr.y, phi2 = pr.z, rho = pr.w;
  const float phv[3] = {phi0, phi1, phi2};
  const float irho = rcp_est(rho);
  // Total distribution f_i = sum_k f_{i,k} of the pulled populations (D
  // stage), in the packed pairs of directions (1, 2), (3, 4) = -(1, 2),
  // (5, 6) and (7, 8) = -(5, 6): on these pairs e_i.v is (v_x, v_y), its
  // negation, (v_x + v_y, v_y - v_x) or its negation, so the collision and
  // the recolouring below run on pairs.
  const int fs = q % 6;
  const float f0 = s.fi0[fs][c];
  const float4 f1234 = s.fi4[fs][0][c], f5678 = s.fi4[fs][1][c];
  const float2 f12 = make_float2(f1234.x, f1234.y), f34 = make_float2(f1234.z, f1234.w);
  const float2 f56 = make_float2(f5678.x, f5678.y), f78 = make_float2(f5678.z, f5678.w);
  // F_s = div T (Eq. 11) as the pair (F_x, F_y) = d_x (T_xx, T_xy) + d_y (T_xy, T_yy);
  // T window column of this node is c + 1.  None with the perturbation
  // operator, whose S is read at the node instead.
  const int tc = c + 1;
  float2 F = make_float2(0.0f, 0.0f);
  float Sxx = 0.0f, Sxy = 0.0f, Syy = 0.0f;
  if (FORCE == 1) {
    const float4 Sc = Tz[tc];
    Sxx = Sc.x;
    Sxy = Sc.y;
    Syy = Sc.w;
  } else {
    // one vector load per stencil node: A = (T_xx, T_xy), B = (T_xy, T_yy)
    const float4 E = Tz[tc + 1], W = Tz[tc - 1], Nn = Tp[tc], S = Tm[tc];
    const float4 NE = Tp[tc + 1], NW = Tp[tc - 1], SE = Tm[tc + 1], SW = Tm[tc - 1];
    auto A = [](const float4& v) { return make_float2(v.x, v.y); };
    auto B = [](const float4& v) { return make_float2(v.z, v.w); };
    const float2 axis = add2(sub2(A(E), A(W)), sub2(B(Nn), B(S)));
    const float2 diag = add2(add2(sub2(A(NE), A(NW)), sub2(A(SE), A(SW))), sub2(add2(B(NE), B(NW)), add2(B(SE), B(SW))));
    F = fma2(bc2(1.0f / 12.0f), diag, mul2(bc2(1.0f / 3.0f), axis));
  }
  // momentum sum_i f_i e_i: (f_1 - f_3, f_2 - f_4) + (f_5 - f_7) (1, 1) + (f_6 - f_8) (-1, 1)
  const float2 d13 = sub2(f12, f34), d57 = sub2(f56, f78);
  const float2 m = add2(d13, make_float2(d57.x - d57.y, d57.x + d57.y));
  // Eq. uk1
  const float2 u = mul2(fma2(bc2(0.5f), F, m), bc2(irho));
  const float ux = u.x, uy = u.y, Fx = F.x, Fy = F.y;
  const int x = x0 + c, y = y0 - 2 + q;
  if (MODE == MODE_FIELDS) {
    const size_t N = static_cast<size_t>(a.nx) * a.ny;
    const size_t idx = static_cast<size_t>(y) * a.nx + x;
    if (a.out_rho) {
      a.out_rho[idx] = phi0 * rho;
      a.out_rho[N + idx] = phi1 * rho;
      a.out_rho[2 * N + idx] = phi2 * rho;
    }
    if (a.out_ux) a.out_ux[idx] = ux;
    if (a.out_uy) a.out_uy[idx] = uy;
    if (a.out_p) a.out_p[idx] = static_cast<double>(rho) / 3.0;
    return;
  }
  // Eqs. vis_1 / tau: 1/nu = sum_k phi_k / nu_k, tau_f = 3 nu + 1/2, omega = 1/tau_f
  const float inu = fmaf(phi0, a.inv_nu[0], fmaf(phi1, a.inv_nu[1], phi2 * a.inv_nu[2]));
  const float om = inu * __fdividef(1.0f, fmaf(0.5f, inu, 3.0f));  // relaxation rate; mass-neutral
  const float g = 1.0f - 0.5f * om;  // Guo prefactor (1 - 1/(2 tau_f))
  const float uu = ux * ux + uy * uy;
  const float uF = ux * Fx + uy * Fy;
  // BGK + Guo (Eqs. 1, 2, 3, 5) written as a correction to f_i, relative to
  // the rest equilibrium w_i rho:
  //   f^dagger_i = f_i + om (w_i rho - f_i) + S_i +- A_i  for the pair (e, -e),
  //   S = w [om rho (4.5 (e.u)^2 - 1.5 u.u) + g (9 (e.u)(e.F) - 3 u.F)]
  //   A = 3 w [om rho (e.u) + g (e.F)].
  // Every term of the correction is small near equilibrium, so an FP32 node
  // at rest is an exact fixed point instead of drifting by an ulp per step.
  const float c0 = -1.5f * om * rho * uu;
  const float c1 = 4.5f * om * rho;
  const float g9 = 9.0f * g;
  const float gm3uF = -3.0f * g * uF;
  const float omr = om * rho;
  // perturbation operator (FORCE 1): Phi_i = om (w_i e_i.S.e_i - B_i tr S),
  // even in e_i, with Leclaire's B_1-4 = 2/27, B_5-8 = 5/108; Phi_0 is the
  // negated sum of the others (-om B_0 tr S in exact arithmetic, as
  // sum_i B_i = 1/3), so the operator moves no mass in FP32 either
  const float trS = Sxx + Syy;
  float phisum = 0.0f;
  float2 fd12, fd34, fd56, fd78;
#pragma unroll
  for (int d = 0; d < 2; ++d) {  // d = 0: axis pairs (1, 2) / (3, 4); d = 1: diagonal pairs (5, 6) / (7, 8)
    const float w = wt(d == 0 ? 1 : 5);
    const float2 eu = d == 0 ? u : make_float2(ux + uy, uy - ux);
    const float2 eF = d == 0 ? F : make_float2(Fx + Fy, Fy - Fx);
    float2 S = mul2(bc2(w), add2(fma2(mul2(bc2(c1), eu), eu, bc2(c0)), fma2(mul2(bc2(g9), eu), eF, bc2(gm3uF))));
    if (FORCE == 1) {
      const float2 eSe = d == 0 ? make_float2(Sxx, Syy) : make_float2(trS + 2.0f * Sxy, trS - 2.0f * Sxy);
      const float Bi = d == 0 ? 2.0f / 27.0f : 5.0f / 108.0f;
      const float2 ph = mul2(bc2(om), fma2(bc2(w), eSe, bc2(-Bi * trS)));
      S = add2(S, ph);
      phisum += 2.0f * ph.x + 2.0f * ph.y;
    }
    const float2 A = mul2(bc2(3.0f * w), fma2(bc2(omr), eu, mul2(bc2(g), eF)));
    const float2 wr = bc2(w * rho);
    const float2 fp = d == 0 ? f12 : f56, fn = d == 0 ? f34 : f78;
    const float2 dp = add2(fp, fma2(bc2(om), sub2(wr, fp), add2(S, A)));
    const float2 dn = add2(fn, fma2(bc2(om), sub2(wr, fn), sub2(S, A)));
    if (d == 0) {
      fd12 = dp;
      fd34 = dn;
    } else {
      fd56 = dp;
      fd78 = dn;
    }
  }
  const float fd0 = f0 + fmaf(om, fmaf(wt(0), rho, -f0), wt(0) * (c0 + gm3uF) - phisum);
  // segregation parameters beta_kl (pairs 12, 13, 23); prod = rho_1 rho_2 rho_3 / rho^3
  const float cb = fminf(a.beta_A * (phi0 * phi1 * phi2), 1.0f);
  const int ns = q % 3;
  const float4 n01 = s.nrm01[ns][c];
  const float2 nn[3] = {make_float2(n01.x, n01.y), make_float2(n01.z, n01.w), s.nrm2[ns][c]};
  float2 R[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int k = p < 2 ? 0 : 1;
    const int l = p == 0 ? 1 : 2;
    const float b = a.beta0 * fmaf(cb, a.beta_h[p], 1.0f);
    const float amp = b * (phv[k] * phv[l]) * rho;  // beta_kl rho_k rho_l / rho
    R[p] = mul2(bc2(amp), nn[p]);
  }
  // V_k = sum_{l != k} beta_kl (rho_k rho_l / rho) n_kl, with n_lk = -n_kl
  const float2 V[3] = {add2(R[0], R[1]), sub2(R[2], R[0]), neg2(add2(R[1], R[2]))};
  // Eq. 6: f^ddagger_{i,k} = phi_k f^dagger_i + w'_i (e_i . V_k), stored at
  // padded column x + 4 and, for the four columns next to each edge, also in
  // the ghost column on the opposite side
  const float2 wa = make_float2(a.wrec[1], a.wrec[2]), wd = make_float2(a.wrec[5], a.wrec[6]);
  float val[27];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 pk = bc2(phv[k]);
    const float2 ta = mul2(wa, V[k]);                                          // e_1.V, e_2.V
    const float2 td = mul2(wd, make_float2(V[k].x + V[k].y, V[k].y - V[k].x));  // e_5.V, e_6.V
    const float2 v12 = fma2(pk, fd12, ta), v34 = fma2(pk, fd34, neg2(ta));
    const float2 v56 = fma2(pk, fd56, td), v78 = fma2(pk, fd78, neg2(td));
    val[plane_of(k, 0)] = phv[k] * fd0;
    val[plane_of(k, 1)] = v12.x;
    val[plane_of(k, 2)] = v12.y;
    val[plane_of(k, 3)] = v34.x;
    val[plane_of(k, 4)] = v34.y;
    val[plane_of(k, 5)] = v56.x;
    val[plane_of(k, 6)] = v56.y;
    val[plane_of(k, 7)] = v78.x;
    val[plane_of(k, 8)] = v78.y;
  }
  const size_t off = static_cast<size_t>(y) * a.pitch + (x + kGhost);
  constexpr int STO = st_out(ST);
  if (STO == ST_RED) {
    // reduced state: phi_k and f^dagger_0 (A), V_kx and f^dagger_1 (X),
    // V_ky and f^dagger_2 (Y), f^dagger_3 .. f^dagger_8; with the ghost
    // copies of the four columns next to each edge as for the populations
    const size_t PS = static_cast<size_t>(a.ny) * a.pitch;
    float4* vo = reinterpret_cast<float4*>(a.fout) + off;
    float* so = a.fout + 4 * kRedVecPlanes * PS + off;
    const float4 A4 = make_float4(phi0, phi1, phi2, fd0);
    const float4 X4 = make_float4(V[0].x, V[1].x, V[2].x, fd12.x);
    const float4 Y4 = make_float4(V[0].y, V[1].y, V[2].y, fd12.y);
    const float sc[6] = {fd34.x, fd34.y, fd56.x, fd56.y, fd78.x, fd78.y};
    auto put = [&](ptrdiff_t d) {
      vo[d] = A4;
      vo[PS + d] = X4;
      vo[2 * PS + d] = Y4;
#pragma unroll
      for (int t = 0; t < 6; ++t) so[t * PS + d] = sc[t];
    };
    put(0);
    if (x < kGhost) put(a.nx);
    if (x >= a.nx - kGhost) put(-static_cast<ptrdiff_t>(a.nx));
  } else if (STO == ST_FP32) {
    // each colour's nine values are stored, with their ghost copies, as soon
    // as they exist: shorter live ranges at the 96-register cap of two CTAs
    // per SM (2.6 % faster than storing all 27 at the end)
    // (a node within kGhost columns of both edges, on grids narrower than
    // 2 kGhost, gets both ghost copies)
    // plane stride in bytes: below 2^32 (checked when a context is created),
    // so each plane's address is one 32 x 32 -> 64-bit multiply-add
    const unsigned psb = static_cast<unsigned>(a.ny) * static_cast<unsigned>(a.pitch) * 4u;
    char* out = reinterpret_cast<char*>(a.fout + off);
    auto st = [psb](char* base, int p, float v) {
      *reinterpret_cast<float*>(base + static_cast<unsigned long long>(p) * psb) = v;
    };
    const bool glo = x < kGhost, ghi = x >= a.nx - kGhost;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int i = 0; i < 9; ++i) st(out, plane_of(k, i), val[plane_of(k, i)]);
      if (glo || ghi) {
        if (glo) {
          char* o2 = out + 4 * static_cast<ptrdiff_t>(a.nx);
#pragma unroll
          for (int i = 0; i < 9; ++i) st(o2, plane_of(k, i), val[plane_of(k, i)]);
        }
        if (ghi) {
          char* o2 = out - 4 * static_cast<ptrdiff_t>(a.nx);
#pragma unroll
          for (int i = 0; i < 9; ++i) st(o2, plane_of(k, i), val[plane_of(k, i)]);
        }
      }
    }
  } else {
    // Encode each colour as rho'_k and 16-bit deviations d_i = f_i - w_i rho_k
    // (rho_k = sum_i f_i): rho'_k absorbs the rounding of the nine d_i, so
    // sum_i (w_i rho'_k + d_i) = rho_k and the colour mass survives storage.
    // Each colour is encoded and stored (with its ghost copies) as soon as
    // its nine values exist, as in the FP32 path; plane strides in bytes as
    // there (a 16-bit plane is half an FP32 plane, below 2 GiB).
    const unsigned psh = static_cast<unsigned>(a.ny) * static_cast<unsigned>(a.pitch) * 2u;
    const unsigned psf = 2u * psh;
    char* dout = reinterpret_cast<char*>(a.dout + off);
    char* rout = reinterpret_cast<char*>(a.rout + off);
    auto st16 = [psh](char* base, int p, unsigned short v) {
      *reinterpret_cast<unsigned short*>(base + static_cast<unsigned long long>(p) * psh) = v;
    };
    auto st32 = [psf](char* base, int p, float v) {
      *reinterpret_cast<float*>(base + static_cast<unsigned long long>(p) * psf) = v;
    };
    const bool glo = x < kGhost, ghi = x >= a.nx - kGhost;
    const ptrdiff_t gh = 2 * static_cast<ptrdiff_t>(a.nx), gf = 4 * static_cast<ptrdiff_t>(a.nx);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float rt = val[plane_of(k, 0)];
#pragma unroll
      for (int i = 1; i < 9; ++i) rt += val[plane_of(k, i)];
      float sr = 0.0f;
      unsigned short code[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        code[i] = enc16<ST>(val[plane_of(k, i)] - wt(i) * rt);
        sr += dec16<ST>(code[i]);
      }
      const float rpk = rt - sr;
#pragma unroll
      for (int i = 0; i < 9; ++i) st16(dout, plane_of(k, i), code[i]);
      st32(rout, k, rpk);
      if (glo || ghi) {
        if (glo) {
#pragma unroll
          for (int i = 0; i < 9; ++i) st16(dout + gh, plane_of(k, i), code[i]);
          st32(rout + gf, k, rpk);
        }
        if (ghi) {
#pragma unroll
          for (int i = 0; i < 9; ++i) st16(dout - gh, plane_of(k, i), code[i]);
          st32(rout - gf, k, rpk);
        }
      }
    }
  }
}

// Every tile is at most kTX columns wide (single grid: strips of kTX and a
// narrower last one; batches: strip_x0() with ceil(nx / kTX) strips), so each
// stage has at most 2 (kTX + 4) = 256 nodes per pair of rows: one per
// consumer thread.
template <int MODE, int ST, int FORCE>
__device__ void consume(Smem& s, const StepArgs& a, int x0, int w, int y0, int h, int tid) {
  constexpr int STI = st_in(ST);
  const int nq = h + 4;  // rows q = 0 .. h+3 <-> y = y0-2 .. y0+h+1
  const RingCols rc = ring_cols(x0);
  volatile int* abort_flag = &s.abort_flag;
  bool dead = false;
  const int J = (h + 3) / 2 + 1;
  for (int j = 0; j < J; ++j) {
    // ---------------- D stage: rows q = 2j, 2j+1 (< nq), columns x0-2 .. x0+w+1
    {
      const int q0 = 2 * j;
      const int nr = min(2, nq - q0);
      if (STI == ST_RED) {
        // march rows q0, q0 + 1 pull from source rows q0 .. q0 + nr + 1; all
        // but the last two were waited for in the previous iteration
        for (int r = j == 0 ? q0 : q0 + 2; r <= q0 + nr + 1 && !dead; ++r) {
          const uint32_t par = static_cast<uint32_t>((r / kRedSlots) & 1);
          if (!mbar_try_wait(&s.full[r % kRedSlots], par))
            dead = !mbar_wait(&s.full[r % kRedSlots], par, abort_flag, a.err);
        }
      } else {
        for (int r = 0; r < nr && !dead; ++r) {
          const int q = q0 + r;
          const uint32_t par = static_cast<uint32_t>((q / kSlots) & 1);
          if (!mbar_try_wait(&s.full[q % kSlots], par)) dead = !mbar_wait(&s.full[q % kSlots], par, abort_flag, a.err);
        }
      }
      if (!dead && tid < nr * (w + 4)) {
        const int W = w + 4;
        const int r = tid >= W ? 1 : 0;
        if (STI == ST_RED)
          stage_density_red(s, a, q0 + r, tid - r * W, w);
        else
          stage_density<STI>(s, q0 + r, tid - r * W, w, rc);
      }
      // this thread is done with the rows of this D stage: the producer may
      // refill their slots (every consumer arrives once per row).  Source
      // rows q0 and q0 + 1 of the reduced state have served all three march
      // rows that pull from them.
      if (STI == ST_RED) {
        mbar_arrive(&s.empty[q0 % kRedSlots]);
        mbar_arrive(&s.empty[(q0 + 1) % kRedSlots]);
      } else {
        for (int r = 0; r < nr; ++r) mbar_arrive(&s.empty[(q0 + r) % kSlots]);
      }
    }
    consumers_sync();
    // ---------------- T stage: rows q = 2j-1, 2j within [1, nq-2], columns x0-1 .. x0+w
    if (!dead) {
      const int qa = max(2 * j - 1, 1), qb = min(2 * j, nq - 2);
      const int nr = qb - qa + 1;
      if (tid < nr * (w + 2)) {  // at most 252 nodes
        const int W = w + 2;
        const int r = tid >= W ? 1 : 0;
        stage_tension<FORCE>(s, a, qa + r, tid - r * W, w);
      }
    }
    consumers_sync();
    // ---------------- C stage: rows q = 2j-2, 2j-1 within [2, h+1], columns x0 .. x0+w-1
    if (!dead) {
      const int qa = max(2 * j - 2, 2), qb = min(2 * j - 1, h + 1);
      const int nr = qb - qa + 1;
      if (tid < nr * w) {  // at most 248 nodes
        const int r = tid >= w ? 1 : 0;
        stage_collide<MODE, ST, FORCE>(s, a, qa + r, tid - r * w, x0, y0);
      }
    }
  }
}

// One tile (strip of w columns starting at x0, rows y0 .. y0+h-1): barrier
// set-up, then the producer warp and the consumer warps.
template <int MODE, int ST, int FORCE, bool STALL = false>
__device__ __forceinline__ void run_tile(Smem& s, const StepArgs& a, const CUtensorMap* map, const CUtensorMap* map1,
                                         int x0, int w, int y0, int h) {
  const int nq = h + 4;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int j = 0; j < kMaxSlots; ++j) {
      mbar_init(&s.full[j], 1);
      mbar_init(&s.empty[j], kConsumers);
    }
    s.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Launched as a programmatic dependent of the previous step (single grid):
  // the next step may be scheduled onto SMs this grid frees, and every CTA
  // waits here, after its set-up, until the previous grid has completed and
  // its writes are visible, before it touches global memory.  Both are no-ops
  // for a launch without that attribute.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (tid >= kConsumers) {
    produce<ST, STALL>(s, a, map, map1, x0, y0, nq, tid - kConsumers);
  } else {
    consume<MODE, ST, FORCE>(s, a, x0, w, y0, h, tid);
  }
}

__device__ __forceinline__ Smem& aligned_smem() {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned: align the block's base
  const uint32_t pad = (128u - (su32(smem_raw) & 127u)) & 127u;
  return *reinterpret_cast<Smem*>(smem_raw + pad);
}

// Single grid: full-width strips of kTX columns and, when kTX does not
// divide nx, a narrower last strip.  CTAs b < full_blocks take full strip
// b % (nx / kTX) and row chunk b / (nx / kTX) of rows_per_cta rows; the
// others take chunks of rows_last rows of the last strip, whose height the
// host picks separately (a narrow CTA costs less per row).  Full-width strips
// with a narrower last one measured 4.6 % faster on a 2048^2 grid than
// equal-width strips (248-node C stages instead of 240).
template <int MODE, int ST, int FORCE, bool STALL = false>
__global__ void __launch_bounds__(kThreads, 2)
    fused_step_kernel(StepArgs a, const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap1) {
  Smem& s = aligned_smem();
  const int nfs = a.nx / kTX;  // full-width strips
  const int b = static_cast<int>(blockIdx.x);
  int strip, y0, h;
  if (b < a.full_blocks) {
    strip = b % nfs;
    y0 = (b / nfs) * a.rows_per_cta;
    h = min(a.rows_per_cta, a.ny - y0);
  } else {
    strip = nfs;
    y0 = (b - a.full_blocks) * a.rows_last;
    h = min(a.rows_last, a.ny - y0);
  }
  const int x0 = strip * kTX;
  const int w = min(kTX, a.nx - x0);
  if (w <= 0 || h <= 0) return;
  run_tile<MODE, ST, FORCE, STALL>(s, a, &tmap, &tmap1, x0, w, y0, h);
}

// Batch of independent grids: CTA b runs work item b (instance, tile); the
// instance's arguments for this step's buffer parity and its tensor maps are
// read from the descriptor in global memory (read-only during the launch).
// The arguments stay there rather than in a shared-memory copy: read from
// shared memory, the compiler keeps the per-instance constants live in
// registers and spills at the 96-register cap of two 288-thread CTAs per
// SM; read from the read-only path they are reloaded at use, as the single
// grid's kernel-parameter constants are (64 % more batch throughput).
// ST: ST_FP32 or ST_RED; ST_F2R takes the descriptors' F2R arguments.
template <int ST>
__global__ void __launch_bounds__(kThreads, 2)
    fused_batch_kernel(const BatchItem* __restrict__ items, const BatchDesc* __restrict__ descs, int parity) {
  Smem& s = aligned_smem();
  const BatchItem it = items[blockIdx.x];
  const BatchDesc* d = descs + it.inst;
  const unsigned char* mp = ST == ST_F2R ? d->map_f2r : d->map[parity];
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(mp);
  const CUtensorMap* map1 = reinterpret_cast<const CUtensorMap*>(mp + 128);
  if (threadIdx.x == kConsumers) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map1))
                 : "memory");
  }
  __syncthreads();
  run_tile<MODE_STEP, ST, 0>(s, ST == ST_F2R ? d->args_f2r[parity] : d->args[parity], map, map1, it.x0, it.w, it.y0,
                             it.h);
}

// Batch whose step arguments travel in the kernel parameter space: the same
// work items and tensor maps, the arguments read from the constant bank.
template <int ST>
__global__ void __launch_bounds__(kThreads, 2)
    fused_batch_param_kernel(const BatchItem* __restrict__ items, const BatchDesc* __restrict__ descs, int parity,
                             const __grid_constant__ BatchArgsBlock args) {
  Smem& s = aligned_smem();
  const BatchItem it = items[blockIdx.x];
  const unsigned char* mp = descs[it.inst].map[parity];
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(mp);
  const CUtensorMap* map1 = reinterpret_cast<const CUtensorMap*>(mp + 128);
  if (threadIdx.x == kConsumers) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map1))
                 : "memory");
  }
  __syncthreads();
  run_tile<MODE_STEP, ST, 0>(s, args.a[it.inst], map, map1, it.x0, it.w, it.y0, it.h);
}

}  // namespace

size_t step_smem_bytes() { return sizeof(Smem) + 128; }

template <int MODE, int ST>
cudaError_t configure_one(int bytes) {
  return cudaFuncSetAttribute(fused_step_kernel<MODE, ST, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t step_configure() {
  const int bytes = static_cast<int>(step_smem_bytes());
  cudaError_t e = configure_one<MODE_STEP, ST_FP32>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_FIELDS, ST_FP32>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_STEP, ST_FP16>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_FIELDS, ST_FP16>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_STEP, ST_BF16>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_FIELDS, ST_BF16>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_STEP, ST_RED>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_FIELDS, ST_RED>(bytes);
  if (e == cudaSuccess) e = configure_one<MODE_STEP, ST_F2R>(bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_step_kernel<MODE_STEP, ST_FP32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_step_kernel<MODE_FIELDS, ST_FP32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_step_kernel<MODE_STEP, ST_FP32, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_batch_kernel<ST_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_batch_kernel<ST_RED>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_batch_kernel<ST_F2R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_batch_param_kernel<ST_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_batch_param_kernel<ST_RED>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_batch(const BatchItem* items, int nitems, const BatchDesc* descs, const BatchArgsBlock* args,
                         int parity, int storage, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const size_t sm = step_smem_bytes();
  if (storage == ST_F2R) {
    fused_batch_kernel<ST_F2R><<<nitems, kThreads, sm, st>>>(items, descs, parity);
  } else if (storage == ST_RED) {
    if (args)
      fused_batch_param_kernel<ST_RED><<<nitems, kThreads, sm, st>>>(items, descs, parity, *args);
    else
      fused_batch_kernel<ST_RED><<<nitems, kThreads, sm, st>>>(items, descs, parity);
  } else if (storage == ST_FP32) {
    if (args)
      fused_batch_param_kernel<ST_FP32><<<nitems, kThreads, sm, st>>>(items, descs, parity, *args);
    else
      fused_batch_kernel<ST_FP32><<<nitems, kThreads, sm, st>>>(items, descs, parity);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int step_occupancy(int* blocks_per_sm) {
  return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, fused_step_kernel<MODE_STEP, ST_FP32, 0>, kThreads, step_smem_bytes()));
}

// A step of the single grid as a programmatic dependent launch: the grid may
// be scheduled while the previous kernel in the stream finishes, and waits in
// run_tile (griddepcontrol.wait) for it to complete.
template <typename... Args>
cudaError_t launch_dependent(void (*kernel)(Args...), int grid, size_t sm, cudaStream_t st, const StepArgs& a,
                             const CUtensorMap& m0, const CUtensorMap& m1) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a, m0, m1);
}

cudaError_t launch_step(const StepArgs& a, const void* tmaps, int grid, int mode, int storage, int force,
                        cudaStream_t st) {
  CUtensorMap m0, m1;
  memcpy(&m0, tmaps, sizeof m0);
  memcpy(&m1, static_cast<const unsigned char*>(tmaps) + 128, sizeof m1);
  const size_t sm = step_smem_bytes();
  if (a.stall_row < 0 && mode == MODE_STEP && force == 0 && (storage == ST_FP32 || storage == ST_RED)) {
    const cudaError_t e = storage == ST_FP32 ? launch_dependent(fused_step_kernel<MODE_STEP, ST_FP32, 0>, grid, sm, st, a, m0, m1)
                                             : launch_dependent(fused_step_kernel<MODE_STEP, ST_RED, 0>, grid, sm, st, a, m0, m1);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  if (a.stall_row >= 0 && mode == MODE_STEP && storage == ST_FP32 && force == 0) {
    // testing hook: the instantiation that can withhold a row
    fused_step_kernel<MODE_STEP, ST_FP32, 0, true><<<grid, kThreads, sm, st>>>(a, m0, m1);
  } else if (force == 1) {  // perturbation operator: FP32 storage only
    if (storage != ST_FP32) return cudaErrorInvalidValue;
    if (mode == MODE_STEP)
      fused_step_kernel<MODE_STEP, ST_FP32, 1><<<grid, kThreads, sm, st>>>(a, m0, m1);
    else
      fused_step_kernel<MODE_FIELDS, ST_FP32, 1><<<grid, kThreads, sm, st>>>(a, m0, m1);
  } else if (storage == ST_FP32) {
    if (mode == MODE_STEP)
      fused_step_kernel<MODE_STEP, ST_FP32, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
    else
      fused_step_kernel<MODE_FIELDS, ST_FP32, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
  } else if (storage == ST_RED) {
    if (mode == MODE_STEP)
      fused_step_kernel<MODE_STEP, ST_RED, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
    else
      fused_step_kernel<MODE_FIELDS, ST_RED, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
  } else if (storage == ST_F2R) {  // FP32 populations in, reduced state out
    if (mode != MODE_STEP) return cudaErrorInvalidValue;
    fused_step_kernel<MODE_STEP, ST_F2R, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
  } else if (storage == ST_FP16) {
    if (mode == MODE_STEP)
      fused_step_kernel<MODE_STEP, ST_FP16, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
    else
      fused_step_kernel<MODE_FIELDS, ST_FP16, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
  } else {
    if (mode == MODE_STEP)
      fused_step_kernel<MODE_STEP, ST_BF16, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
    else
      fused_step_kernel<MODE_FIELDS, ST_BF16, 0><<<grid, kThreads, sm, st>>>(a, m0, m1);
  }
  return cudaGetLastError();
}

size_t population_bytes(int nx, int ny, int storage) {
  const size_t PS = static_cast<size_t>(pitch_of(nx)) * static_cast<size_t>(ny);
  if (storage == ST_RED) return (4 * kRedVecPlanes + kRedSclPlanes) * PS * 4;
  return storage == ST_FP32 ? 27 * PS * 4 : 27 * PS * 2 + 3 * PS * 4;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder(cudaError_t* err) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  *err = cudaSuccess;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    if (q != cudaDriverEntryPointSuccess || !fn) {
      *err = cudaErrorNotSupported;
      return nullptr;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

cudaError_t encode_3d(PFN_cuTensorMapEncodeTiled_v12000 encode, void* tmap, CUtensorMapDataType type, int esize,
                      const void* base, int P, int ny, int planes, int boxw, int boxp) {
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(P), static_cast<cuuint64_t>(ny),
                              static_cast<cuuint64_t>(planes)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(P) * esize, static_cast<cuuint64_t>(ny) * P * esize};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(boxw), 1, static_cast<cuuint32_t>(boxp)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(tmap), type, 3, const_cast<void*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t encode_population_maps(void* tmaps, const void* buf, int nx, int ny, int storage) {
  cudaError_t e;
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder(&e);
  if (!encode) return e;
  const int P = pitch_of(nx);
  unsigned char* m = static_cast<unsigned char*>(tmaps);
  if (storage == ST_RED) {
    // the float4 planes as a (16, P/4, ny, 3) FP32 tensor (four columns of
    // float4 innermost: 64-byte inner runs rather than 16-byte ones), box
    // (16, kPW/4, 1, 3) at column tma_x/4; the scalar planes as (P, ny, 6),
    // box (kPW, 1, 6).  P and tma_x are multiples of 4.
    const cuuint64_t dims[4] = {16, static_cast<cuuint64_t>(P / 4), static_cast<cuuint64_t>(ny), kRedVecPlanes};
    const cuuint64_t strides[3] = {64, static_cast<cuuint64_t>(P) * 16, static_cast<cuuint64_t>(ny) * P * 16};
    const cuuint32_t box[4] = {16, static_cast<cuuint32_t>(kPW / 4), 1, kRedVecPlanes};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(m), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                              const_cast<void*>(buf), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const float* scl = static_cast<const float*>(buf) + static_cast<size_t>(4 * kRedVecPlanes) * P * ny;
    return encode_3d(encode, m + 128, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, scl, P, ny, kRedSclPlanes, kPW,
                     kRedSclPlanes);
  }
  if (storage == ST_FP32) {
    e = encode_3d(encode, m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, buf, P, ny, 27, kPW, 9);
    if (e == cudaSuccess) memcpy(m + 128, m, 128);  // unused second map
    return e;
  }
  const size_t PS = static_cast<size_t>(P) * ny;
  const float* rho = reinterpret_cast<const float*>(static_cast<const unsigned short*>(buf) + 27 * PS);
  e = encode_3d(encode, m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, buf, P, ny, 27, kDevBoxCols, 9);
  if (e == cudaSuccess) e = encode_3d(encode, m + 128, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, rho, P, ny, 3, kPW, 3);
  return e;
}

}  // namespace lbm3
