// Internal declarations of the reverse-mode (adjoint) kernels of liblbm3.
// Nothing here is part of the public C ABI (see include/lbm3.h).
#pragma once

#include "lbm3_internal.h"

namespace lbm3 {

// ------------------------------------------------------ reverse mode
// Scratch of the adjoint step, carved from one allocation of
// adj_scratch_floats(N) floats: two cotangent buffers of a stored state
// ([27][N] each, ping-pong), the cotangents of f_i [9][N], rho_k [3][N],
// grad phi_k [6][N] and F_s [2][N], and the recomputed rho_k [3][N],
// grad phi_k [6][N] and T [3][N] of the state being differentiated.
struct AdjBuffers {
  float* lam[2];
  float* lam9;
  float* lamr;
  float* lamg;
  float* lamF;
  float* rho3;
  float* gphi;
  float* T;
};
size_t adj_scratch_floats(int N);
void adj_layout(float* base, int N, AdjBuffers* b);
int adj_blocks(int N);  // rows of the FP64 accumulator [blocks][6]: dJ/dsigma (0..2), dJ/dh (3..5)
// colour fractions phi_k (FP64 [3][N]) of a stored FP32 state
cudaError_t launch_phi(const float* st, double* phi, int nx, int ny, cudaStream_t s);
// cotangent of the final stored state from dJ/dphi (FP64 [3][N]) into b.lam[lam_out]
cudaError_t launch_adj_seed(const float* st_final, const double* dphi, const AdjBuffers& b, int lam_out, int nx,
                            int ny, cudaStream_t s);
// one adjoint step: b.lam[lam_in] = dJ/dS_t -> b.lam[lam_in ^ 1] = dJ/dS_{t-1}, st_prev = S_{t-1}
cudaError_t launch_adj_step(const float* st_prev, const StepArgs& a, const AdjBuffers& b, int lam_in, double* acc,
                            cudaStream_t s);
// dJ/df (post-streaming populations, planes plane0.., FP64) and dJ/drho_k of a rest-equilibrium start
cudaError_t launch_adj_dpop(const float* lam, double* out, int nx, int ny, int plane0, int nplanes, cudaStream_t s);
cudaError_t launch_adj_drho(const float* lam, double* out, int nx, int ny, cudaStream_t s);

}  // namespace lbm3
