// Internal declarations of the reverse-mode (adjoint) kernels of liblbm3.
// Nothing here is part of the public C ABI (see include/lbm3.h).
#pragma once

#include "lbm3_internal.h"

namespace lbm3 {

// ------------------------------------------------------ reverse mode
// Scratch of the adjoint, carved from one allocation of adj_scratch_floats(N)
// floats.  Cotangents of the pulled populations of a step, factored as
// dJ/df_ik = lam9_i + lamr_k ([9][N] and [3][N], ping-pong between steps);
// of grad phi_k [6][N] and F_s [2][N]; and the recomputed rho_k [3][N],
// grad phi_k [6][N] and T [3][N] of the state being differentiated and of the
// next one (two slots).
struct AdjBuffers {
  float* lam9[2];
  float* lamr[2];
  float* lamg;
  float* lamF;
  float* rho3[2];
  float* gphi[2];
  float* T[2];
};
size_t adj_scratch_floats(int N);
void adj_layout(float* base, int N, AdjBuffers* b);
int adj_blocks(int N);  // rows of the FP64 accumulator [blocks][6]: dJ/dsigma (0..2), dJ/dh (3..5)
// colour fractions phi_k (FP64 [3][N]) of a stored FP32 state
cudaError_t launch_phi(const float* st, double* phi, int nx, int ny, cudaStream_t s);
// cotangent (lam9[lam], lamr[lam]) of the pulled populations at the end of
// the run from dJ/dphi (FP64 [3][N]); uses rho3[1] as scratch
cudaError_t launch_adj_seed(const float* st_final, const double* dphi, const AdjBuffers& b, int lam, int nx, int ny,
                            cudaStream_t s);
// rho3, gphi and T of state st into slot `slot`
cudaError_t launch_adj_fields(const float* st, const StepArgs& a, const AdjBuffers& b, int slot, cudaStream_t s);
// one adjoint step (three launches): st_prev = S_{t-1} with its fields in
// slot `slot`, cotangent in lam -> cotangent of step t-1's pulled
// populations in lam ^ 1; when st_next (= S_{t-2}) is given, its fields are
// computed into slot ^ 1 alongside
cudaError_t launch_adj_step(const float* st_prev, const float* st_next, const StepArgs& a, const AdjBuffers& b,
                            int slot, int lam, double* acc, cudaStream_t s);
// dJ/df (post-streaming populations at t = 0, planes plane0.., FP64) and
// dJ/drho_k of a rest-equilibrium start, from the cotangent in lam
cudaError_t launch_adj_dpop(const AdjBuffers& b, int lam, double* out, int nx, int ny, int plane0, int nplanes,
                            cudaStream_t s);
cudaError_t launch_adj_drho(const AdjBuffers& b, int lam, double* out, int nx, int ny, cudaStream_t s);

}  // namespace lbm3
