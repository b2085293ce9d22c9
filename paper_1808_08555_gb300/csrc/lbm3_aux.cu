// Auxiliary kernels of liblbm3: state set-up and read-out in the pull layout,
// and the FP64 mass/momentum reductions (over the library's padded layout,
// and over a plain [27][ny][nx] array for the allocation-free entry point).
//
// The library stores, between steps, the post-collision populations
// f^ddagger_{i,k}(x) at the node x where they were produced (before
// streaming).  The post-streaming state the paper works with (Eq. 30) is then
// f_{i,k}(x, t) = stored_{i,k}(x - e_i); these kernels translate between the
// two.

#include <cmath>
#include <cstdint>

#include "lbm3_internal.h"

namespace lbm3 {
namespace {

__device__ __forceinline__ int wrapi(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ int dir_ex(int i) { return ex(i); }
__device__ __forceinline__ int dir_ey(int i) { return ey(i); }

// Padded, group-ordered layout (see lbm3_internal.h): plane p of direction
// i, row y, padded column xp holds the value of node x = (xp - 4) mod nx.

// stored_{i,k}(x) = w_i rho_k(x + e_i): the rest equilibrium w_i rho_k after
// the pull of the next step.
__global__ void init_from_rho_kernel(const double* __restrict__ rho, float* __restrict__ f, int nx, int ny) {
  const int plane = blockIdx.z;  // k*9 + i (input numbering)
  const int k = plane / 9, i = plane % 9;
  const int P = pitch_of(nx);
  const size_t N = static_cast<size_t>(nx) * ny;
  float* dst = f + static_cast<size_t>(plane_of(k, i)) * P * ny;
  const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    const size_t row = static_cast<size_t>(wrapi(y + dir_ey(i), ny)) * nx;
    for (int xp = blockIdx.x * blockDim.x + threadIdx.x; xp < P; xp += gridDim.x * blockDim.x) {
      const int x = wrapi(xp - kGhost, nx);
      dst[static_cast<size_t>(y) * P + xp] = static_cast<float>(w * rho[k * N + row + wrapi(x + dir_ex(i), nx)]);
    }
  }
}

// stored(x) = fpost(x + e_i) for input planes plane0 .. plane0+nplanes-1
// (fpost numbered k*9 + i, unpadded).
__global__ void set_planes_kernel(const double* __restrict__ fpost, float* __restrict__ f, int nx, int ny,
                                  int plane0) {
  const int pl = blockIdx.z;
  const int plane = plane0 + pl, k = plane / 9, i = plane % 9;
  const int P = pitch_of(nx);
  const size_t N = static_cast<size_t>(nx) * ny;
  float* dst = f + static_cast<size_t>(plane_of(k, i)) * P * ny;
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    const size_t row = static_cast<size_t>(wrapi(y + dir_ey(i), ny)) * nx;
    for (int xp = blockIdx.x * blockDim.x + threadIdx.x; xp < P; xp += gridDim.x * blockDim.x) {
      const int x = wrapi(xp - kGhost, nx);
      dst[static_cast<size_t>(y) * P + xp] = static_cast<float>(fpost[pl * N + row + wrapi(x + dir_ex(i), nx)]);
    }
  }
}

// fpost(x) = stored(x - e_i), written unpadded with numbering k*9 + i.
__global__ void get_planes_kernel(const float* __restrict__ f, double* __restrict__ fpost, int nx, int ny,
                                  int plane0) {
  const int pl = blockIdx.z;
  const int plane = plane0 + pl, k = plane / 9, i = plane % 9;
  const int P = pitch_of(nx);
  const size_t N = static_cast<size_t>(nx) * ny;
  const float* src = f + static_cast<size_t>(plane_of(k, i)) * static_cast<size_t>(P) * ny;
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    const size_t srow = static_cast<size_t>(wrapi(y - dir_ey(i), ny)) * P;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x)
      fpost[pl * N + static_cast<size_t>(y) * nx + x] = static_cast<double>(src[srow + wrapi(x - dir_ex(i), nx) + kGhost]);
  }
}

// ------------------------------------------------------------------ 16-bit
// FP32 padded stored values (as the FP32 layout) -> rho' and 16-bit
// deviations, per padded node, with the same arithmetic as the step's encode.
template <int ST>
__global__ void encode_kernel(const float* __restrict__ f, unsigned short* __restrict__ dev, int nx, int ny) {
  const size_t PS = static_cast<size_t>(pitch_of(nx)) * ny;
  float* rho = reinterpret_cast<float*>(dev + 27 * PS);
  for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < PS;
       n += static_cast<size_t>(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float v[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) v[i] = f[plane_of(k, i) * PS + n];
      float rt = v[0];
#pragma unroll
      for (int i = 1; i < 9; ++i) rt += v[i];
      float sr = 0.0f;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const unsigned short b = enc16<ST>(v[i] - wt(i) * rt);
        dev[plane_of(k, i) * PS + n] = b;
        sr += dec16<ST>(b);
      }
      rho[k * PS + n] = rt - sr;
    }
  }
}

template <int ST>
__global__ void decode_kernel(const unsigned short* __restrict__ dev, float* __restrict__ f, int nx, int ny) {
  const size_t PS = static_cast<size_t>(pitch_of(nx)) * ny;
  const float* rho = reinterpret_cast<const float*>(dev + 27 * PS);
  for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < PS;
       n += static_cast<size_t>(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float r = rho[k * PS + n];
#pragma unroll
      for (int i = 0; i < 9; ++i)
        f[plane_of(k, i) * PS + n] = fmaf(wt(i), r, dec16<ST>(dev[plane_of(k, i) * PS + n]));
    }
  }
}

// FP32 stored populations (padded, group-ordered layout) of a reduced state:
// the value of colour k, direction i at node x is Eq. 6 formed from x's own
// phi_k, f^dagger_i and V_k by red_pop, as the step's C stage forms it for
// the FP32 storage (so the expansion is bit-identical to that storage).
// Ghost columns are expanded from the reduced state's ghost columns.
__global__ void expand_red_kernel(const float* __restrict__ red, float* __restrict__ f, int nx, int ny,
                                  StepArgs a) {
  const int P = pitch_of(nx);
  const size_t PS = static_cast<size_t>(P) * ny;
  const float4* vec = reinterpret_cast<const float4*>(red);
  const float* scl = red + 4 * kRedVecPlanes * PS;
  for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < PS;
       n += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (static_cast<int>(n % P) >= nx + 2 * kGhost) continue;  // columns after the right ghosts are unused
    const float4 A = vec[n], X = vec[PS + n], Y = vec[2 * PS + n];
    const float fd[9] = {A.w, X.w, Y.w, scl[n], scl[PS + n], scl[2 * PS + n], scl[3 * PS + n], scl[4 * PS + n],
                         scl[5 * PS + n]};
    const float ph[3] = {A.x, A.y, A.z}, vx[3] = {X.x, X.y, X.z}, vy[3] = {Y.x, Y.y, Y.z};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 9; ++i) f[plane_of(k, i) * PS + n] = red_pop(i, ph[k], fd[i], vx[k], vy[k], a.wrec);
  }
}

__global__ void check_rho_kernel(const double* __restrict__ rho, int n, unsigned int* bad) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double a = rho[j], b = rho[n + j], c = rho[2 * n + j];
    const bool ok = std::isfinite(a) && std::isfinite(b) && std::isfinite(c) && a >= 0.0 && b >= 0.0 &&
                    c >= 0.0 && (a + b + c) > 0.0;
    if (!ok) atomicOr(bad, 1u);
  }
}

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-level FP64 sums of (mass_r, mass_g, mass_b, mom_x, mom_y) over nodes:
// per thread in registers, then warp shuffles, then one shared-memory pass.
__global__ void reduce_partial_kernel(const float* __restrict__ f, int N, double* __restrict__ partial) {
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const double v = static_cast<double>(f[static_cast<size_t>(k * 9 + i) * N + n]);
        acc[k] += v;
        acc[3] += v * ex(i);
        acc[4] += v * ey(i);
      }
    }
  }
  __shared__ double red[kRedThreads / 32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const double v = warp_sum(acc[j]);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      double v = lane < kRedThreads / 32 ? red[lane][j] : 0.0;
      v = warp_sum(v);
      if (lane == 0) partial[blockIdx.x * 5 + j] = v;
    }
  }
}

// Same sums over the library's padded, group-ordered layout (ghost columns
// excluded).
__global__ void reduce_partial_padded_kernel(const float* __restrict__ f, int nx, int ny,
                                             double* __restrict__ partial) {
  const int P = pitch_of(nx);
  const int N = nx * ny;
  const size_t NP = static_cast<size_t>(P) * ny;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const size_t off = static_cast<size_t>(n / nx) * P + (n % nx) + kGhost;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const double v = static_cast<double>(f[static_cast<size_t>(plane_of(k, i)) * NP + off]);
        acc[k] += v;
        acc[3] += v * ex(i);
        acc[4] += v * ey(i);
      }
    }
  }
  __shared__ double red[kRedThreads / 32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const double v = warp_sum(acc[j]);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      double v = lane < kRedThreads / 32 ? red[lane][j] : 0.0;
      v = warp_sum(v);
      if (lane == 0) partial[blockIdx.x * 5 + j] = v;
    }
  }
}

// Same sums over 16-bit deviation storage (values rebuilt as w_i rho' + d).
template <int ST>
__global__ void reduce_partial_dev_kernel(const unsigned short* __restrict__ dev, int nx, int ny,
                                          double* __restrict__ partial) {
  const int P = pitch_of(nx);
  const int N = nx * ny;
  const size_t PS = static_cast<size_t>(P) * ny;
  const float* rho = reinterpret_cast<const float*>(dev + 27 * PS);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const size_t off = static_cast<size_t>(n / nx) * P + (n % nx) + kGhost;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float r = rho[k * PS + off];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const double v = static_cast<double>(fmaf(wt(i), r, dec16<ST>(dev[plane_of(k, i) * PS + off])));
        acc[k] += v;
        acc[3] += v * ex(i);
        acc[4] += v * ey(i);
      }
    }
  }
  __shared__ double red[kRedThreads / 32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const double v = warp_sum(acc[j]);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      double v = lane < kRedThreads / 32 ? red[lane][j] : 0.0;
      v = warp_sum(v);
      if (lane == 0) partial[blockIdx.x * 5 + j] = v;
    }
  }
}

__global__ void reduce_final_kernel(const double* __restrict__ partial, int blocks, double* __restrict__ out) {
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < blocks; b += blockDim.x)
#pragma unroll
    for (int j = 0; j < 5; ++j) acc[j] += partial[b * 5 + j];
  __shared__ double red[kRedThreads / 32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const double v = warp_sum(acc[j]);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      double v = lane < kRedThreads / 32 ? red[lane][j] : 0.0;
      v = warp_sum(v);
      if (lane == 0) out[j] = v;
    }
  }
}

int grid_for(size_t N) {
  const size_t b = (N + 255) / 256;
  return static_cast<int>(b < 65535 ? (b > 0 ? b : 1) : 65535);
}

// Plane kernels: 256 threads along a row's columns, rows by blockIdx.y (at
// most 1024 per grid stride), one plane per blockIdx.z.
dim3 plane_grid(int cols, int ny, int planes) {
  return dim3(static_cast<unsigned>((cols + 255) / 256), static_cast<unsigned>(ny < 1024 ? ny : 1024),
              static_cast<unsigned>(planes));
}

}  // namespace

cudaError_t launch_init_from_rho(const double* rho, float* f, int nx, int ny, cudaStream_t s) {
  init_from_rho_kernel<<<plane_grid(pitch_of(nx), ny, 27), 256, 0, s>>>(rho, f, nx, ny);
  return cudaGetLastError();
}

cudaError_t launch_set_planes(const double* fpost, float* f, int nx, int ny, int plane0, int nplanes,
                              cudaStream_t s) {
  set_planes_kernel<<<plane_grid(pitch_of(nx), ny, nplanes), 256, 0, s>>>(fpost, f, nx, ny, plane0);
  return cudaGetLastError();
}

cudaError_t launch_get_planes(const float* f, double* fpost, int nx, int ny, int plane0, int nplanes,
                              cudaStream_t s) {
  get_planes_kernel<<<plane_grid(nx, ny, nplanes), 256, 0, s>>>(f, fpost, nx, ny, plane0);
  return cudaGetLastError();
}

cudaError_t launch_check_rho(const double* rho, int n, unsigned int* bad, cudaStream_t s) {
  check_rho_kernel<<<grid_for(static_cast<size_t>(n)), 256, 0, s>>>(rho, n, bad);
  return cudaGetLastError();
}

int reduce_blocks(int N) {
  int b = (N + kRedThreads * 8 - 1) / (kRedThreads * 8);
  return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

cudaError_t launch_reduce(const float* f, int N, double* partial, int blocks, double* out, cudaStream_t s) {
  reduce_partial_kernel<<<blocks, kRedThreads, 0, s>>>(f, N, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_final_kernel<<<1, kRedThreads, 0, s>>>(partial, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_padded(const float* f, int nx, int ny, double* partial, int blocks, double* out,
                                 cudaStream_t s) {
  reduce_partial_padded_kernel<<<blocks, kRedThreads, 0, s>>>(f, nx, ny, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_final_kernel<<<1, kRedThreads, 0, s>>>(partial, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_encode(const float* fp32, void* buf, int nx, int ny, int storage, cudaStream_t s) {
  const int g = grid_for(static_cast<size_t>(pitch_of(nx)) * ny);
  unsigned short* d = static_cast<unsigned short*>(buf);
  if (storage == ST_FP16)
    encode_kernel<ST_FP16><<<g, 256, 0, s>>>(fp32, d, nx, ny);
  else
    encode_kernel<ST_BF16><<<g, 256, 0, s>>>(fp32, d, nx, ny);
  return cudaGetLastError();
}

cudaError_t launch_expand_reduced(const float* red, float* fp32, int nx, int ny, const StepArgs& a,
                                  cudaStream_t s) {
  const int g = grid_for(static_cast<size_t>(pitch_of(nx)) * ny);
  expand_red_kernel<<<g, 256, 0, s>>>(red, fp32, nx, ny, a);
  return cudaGetLastError();
}

cudaError_t launch_decode(const void* buf, float* fp32, int nx, int ny, int storage, cudaStream_t s) {
  const int g = grid_for(static_cast<size_t>(pitch_of(nx)) * ny);
  const unsigned short* d = static_cast<const unsigned short*>(buf);
  if (storage == ST_FP16)
    decode_kernel<ST_FP16><<<g, 256, 0, s>>>(d, fp32, nx, ny);
  else
    decode_kernel<ST_BF16><<<g, 256, 0, s>>>(d, fp32, nx, ny);
  return cudaGetLastError();
}

cudaError_t launch_reduce_dev(const void* buf, int nx, int ny, int storage, double* partial, int blocks,
                              double* out, cudaStream_t s) {
  const unsigned short* d = static_cast<const unsigned short*>(buf);
  if (storage == ST_FP16)
    reduce_partial_dev_kernel<ST_FP16><<<blocks, kRedThreads, 0, s>>>(d, nx, ny, partial);
  else
    reduce_partial_dev_kernel<ST_BF16><<<blocks, kRedThreads, 0, s>>>(d, nx, ny, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_final_kernel<<<1, kRedThreads, 0, s>>>(partial, blocks, out);
  return cudaGetLastError();
}

}  // namespace lbm3
