// Host side of liblbm3: the C ABI declared in include/lbm3.h.
//
// The context owns (or borrows) two FP32 population buffers used in
// ping-pong: one holds the current state (post-collision populations stored
// where they were produced, read by the next step's pull), the other is the
// target of the next step and, between steps, doubles as staging memory for
// host input/output, so no extra full-grid allocation is made.  Each buffer
// has a TMA tensor descriptor, encoded once when the buffer is set.

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm3.h"
#include "lbm3_adjoint.h"
#include "lbm3_internal.h"

using lbm3::StepArgs;

struct lbm3_ctx {
  lbm3_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int occ = 0;
  float* buf[2] = {nullptr, nullptr};
  bool owns_bufs = false;
  int cur = 0;
  bool state_set = false;
  int64_t t = 0;
  size_t buf_bytes = 0;
  // small scratch: reduction partials, reduction output, error word, check flag
  unsigned char* scratch = nullptr;
  double* partial = nullptr;
  double* red_out = nullptr;
  unsigned int* err = nullptr;
  unsigned int* bad = nullptr;
  int red_blocks = 1;
  int rows_override = 0;
  int stall_row = -1;  // lbm3_debug_stall_row: applies to the next lbm3_step launch only
  StepArgs base{};
  // TMA descriptors of buf[0] and buf[1]: one (FP32) or two (deviations, rho')
  alignas(64) unsigned char tmap[2][256];
  float* shadow = nullptr;  // 16-bit and reduced storage: FP32 populations for host I/O
  alignas(64) unsigned char shadow_map[256];  // its TMA descriptors (reduced storage)
  bool in_shadow = false;   // reduced storage: the state is the FP32 populations in the shadow
  double* diag = nullptr;   // interface diagnostics: block partial sums and totals (first use)
  // reverse mode: checkpoints S_0, S_K, S_2K, ... of a recorded run, the
  // recomputed states of one segment, the adjoint scratch and accumulator
  unsigned char* ckpt = nullptr;
  size_t ckpt_slots = 0;
  unsigned char* tape = nullptr;
  size_t tape_slots = 0;
  std::vector<unsigned char> ckpt_maps;  // 256 bytes of TMA descriptors per slot
  std::vector<unsigned char> tape_maps;
  float* adj = nullptr;
  double* acc = nullptr;
  int64_t tape_steps = 0;
  int tape_every = 0;
  bool tape_valid = false;
  std::string msg;
};

namespace {

const char* kNullCtxMsg = "lbm3: NULL context";

lbm3_status fail(lbm3_ctx* c, lbm3_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->msg = buf;
  return st;
}

lbm3_status cuda_fail(lbm3_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LBM3_ECUDA, "lbm3: %s: %s", where, cudaGetErrorString(e));
}

#define LBM3_CUDA(ctx, call)                                 \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

size_t nodes(const lbm3_params& p) { return static_cast<size_t>(p.nx) * static_cast<size_t>(p.ny); }

// one population buffer: 27 planes of ny rows with the padded pitch nx + 8
size_t buffer_bytes(const lbm3_params& p) { return lbm3::population_bytes(p.nx, p.ny, p.storage); }

size_t fp32_bytes(const lbm3_params& p) { return lbm3::population_bytes(p.nx, p.ny, LBM3_FP32); }

lbm3_status validate(const lbm3_params* p, std::string* why) {
  char b[256];
  if (!p) {
    *why = "lbm3: NULL params";
    return LBM3_EINVAL;
  }
  if (p->nx < 4 || p->nx % 4 != 0 || p->ny < 1) {
    std::snprintf(b, sizeof b, "lbm3: grid %d x %d: nx must be a multiple of 4 and >= 4, ny >= 1", p->nx, p->ny);
    *why = b;
    return LBM3_EINVAL;
  }
  if (static_cast<double>(p->nx) * p->ny >= 2147483648.0) {
    *why = "lbm3: nx*ny must be below 2^31";
    return LBM3_EINVAL;
  }
  // the step kernel addresses a population plane with a 32-bit byte stride
  if (static_cast<double>(lbm3::pitch_of(p->nx)) * p->ny * 4.0 >= 4294967296.0) {
    std::snprintf(b, sizeof b, "lbm3: grid %d x %d: one padded FP32 plane (%d x %d x 4 bytes) must be below 4 GiB",
                  p->nx, p->ny, lbm3::pitch_of(p->nx), p->ny);
    *why = b;
    return LBM3_EINVAL;
  }
  for (int k = 0; k < 3; ++k) {
    if (!(p->tau[k] > 0.5) || !std::isfinite(p->tau[k])) {
      std::snprintf(b, sizeof b, "lbm3: tau[%d] = %g must be > 0.5", k, p->tau[k]);
      *why = b;
      return LBM3_EINVAL;
    }
    if (!(p->rho0[k] > 0.0) || !std::isfinite(p->rho0[k])) {
      std::snprintf(b, sizeof b, "lbm3: rho0[%d] = %g must be > 0", k, p->rho0[k]);
      *why = b;
      return LBM3_EINVAL;
    }
  }
  const double s[3] = {p->sigma12, p->sigma13, p->sigma23};
  for (int q = 0; q < 3; ++q)
    if (!(s[q] > 0.0) || !std::isfinite(s[q])) {
      *why = "lbm3: every sigma_kl must be > 0";
      return LBM3_EINVAL;
    }
  if (!(p->beta0 > 0.0 && p->beta0 <= 1.0)) {
    *why = "lbm3: beta0 must be in (0, 1]";
    return LBM3_EINVAL;
  }
  if (p->beta_form < 0 || p->beta_form > 3 || p->recolor_form < 0 || p->recolor_form > 1 ||
      p->storage < LBM3_FP32 || p->storage > LBM3_REDUCED || p->force_form < 0 || p->force_form > 1) {
    *why = "lbm3: beta_form, recolor_form, storage or force_form out of range";
    return LBM3_EINVAL;
  }
  if (!(p->normal_delta >= 0.0 && p->normal_delta <= 1.0)) {
    *why = "lbm3: normal_delta must be in [0, 1]";
    return LBM3_EINVAL;
  }
  if (p->force_form == LBM3_FORCE_PERTURBATION && p->storage != LBM3_FP32) {
    *why = "lbm3: the perturbation-operator force form needs FP32 storage";
    return LBM3_EINVAL;
  }
  return LBM3_OK;
}

// Eq. 20
double g_of_X(double X) {
  if (X < -1.0) return 1.0;
  if (X < 0.0) return 1.0 - std::sqrt(1.0 - X * X);
  if (X <= 1.0) return std::sqrt(1.0 - X * X) - 1.0;
  return -1.0;
}

// Host-side constants of the step: 1/nu_k, the C_kl prefactor, sigmas, the
// per-pair beta coefficients and the recolouring direction weights.
void fill_constants(const lbm3_params& p, StepArgs* a) {
  const double s[3] = {p.sigma12, p.sigma13, p.sigma23};
  const int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2};
  auto sig = [&](int k, int l) {
    const int lo = k < l ? k : l, hi = k < l ? l : k;
    return lo == 0 ? (hi == 1 ? s[0] : s[1]) : s[2];
  };
  double X[3], ang[3];
  bool tri = true;
  for (int q = 0; q < 3; ++q) {
    const int k = pk[q], l = pl[q], m = 3 - k - l;
    const double smk = sig(m, k), sml = sig(m, l), skl = sig(k, l);
    X[q] = (smk * smk + sml * sml - skl * skl) / (2.0 * smk * sml);  // Eq. 18
    tri = tri && std::fabs(X[q]) < 1.0;
    ang[q] = std::acos(X[q] < -1.0 ? -1.0 : (X[q] > 1.0 ? 1.0 : X[q]));
  }
  double A = 0.0, h[3] = {0.0, 0.0, 0.0};
  switch (p.beta_form) {
    case LBM3_BETA_PAPER:  // Eqs. 19-20
      A = 35.0;
      for (int q = 0; q < 3; ++q) h[q] = g_of_X(X[q]);
      break;
    case LBM3_BETA_FU:  // Eq. fu
      break;
    case LBM3_BETA_SPENCER:  // Eq. 16; beta^0 everywhere without a Neumann triangle
      if (tri) {
        A = 27.0;
        h[1] = std::sin(ang[2]) - 1.0;
        h[2] = std::sin(ang[1]) - 1.0;
      }
      break;
    case LBM3_BETA_LECLAIRE:  // Eq. 17; beta^0 everywhere without a Neumann triangle
      if (tri) {
        A = 35.0;
        int qm = 0;
        for (int q = 1; q < 3; ++q)
          if (ang[q] > ang[qm]) qm = q;
        const double pi = std::acos(-1.0);
        for (int q = 0; q < 3; ++q) h[q] = q == qm ? 0.0 : std::sin(pi - ang[qm] - ang[q]) - 1.0;
      }
      break;
  }
  for (int k = 0; k < 3; ++k) a->inv_nu[k] = static_cast<float>(3.0 / (p.tau[k] - 0.5));
  for (int q = 0; q < 3; ++q) {
    a->cpair[q] = static_cast<float>(1e6 / (p.rho0[pk[q]] * p.rho0[pl[q]]));
    a->sigma[q] = static_cast<float>(s[q]);
    a->beta_h[q] = static_cast<float>(h[q]);
  }
  a->beta0 = static_cast<float>(p.beta0);
  a->beta_A = static_cast<float>(A);
  a->ndelta = static_cast<float>(p.normal_delta);
  for (int i = 0; i < 9; ++i) {
    const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const double len = std::sqrt(static_cast<double>(lbm3::ex(i) * lbm3::ex(i) + lbm3::ey(i) * lbm3::ey(i)));
    a->wrec[i] = static_cast<float>((p.recolor_form == LBM3_RECOLOR_COSINE && i != 0) ? w / len : w);
  }
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

lbm3_status encode_maps(lbm3_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    const cudaError_t e = lbm3::encode_population_maps(c->tmap[b], c->buf[b], c->p.nx, c->p.ny, c->p.storage);
    if (e != cudaSuccess) return cuda_fail(c, e, "encoding the TMA descriptor of a population buffer");
  }
  return LBM3_OK;
}

lbm3_status ensure_buffers(lbm3_ctx* c) {
  if (c->buf[0]) return LBM3_OK;
  void* a = nullptr;
  void* b = nullptr;
  if (cudaMalloc(&a, c->buf_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LBM3_ENOMEM, "lbm3: cannot allocate %zu bytes for populations", c->buf_bytes);
  }
  if (cudaMalloc(&b, c->buf_bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(a);
    return fail(c, LBM3_ENOMEM, "lbm3: cannot allocate %zu bytes for populations", c->buf_bytes);
  }
  c->buf[0] = static_cast<float*>(a);
  c->buf[1] = static_cast<float*>(b);
  c->owns_bufs = true;
  return encode_maps(c);
}

// FP32 target of host input: the current buffer, or for the 16-bit and
// reduced storages the FP32 shadow (allocated on first use).  A 16-bit
// storage encodes it into the current buffer; the reduced storage keeps the
// state there until the next step, which reads it as FP32 populations and
// writes the reduced state (the reduced state holds only populations that a
// step has produced).
lbm3_status fp32_target(lbm3_ctx* c, float** out) {
  if (c->p.storage == LBM3_FP32) {
    *out = c->buf[c->cur];
    return LBM3_OK;
  }
  if (!c->shadow) {
    void* p = nullptr;
    if (cudaMalloc(&p, fp32_bytes(c->p)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, LBM3_ENOMEM, "lbm3: cannot allocate the FP32 shadow of the populations");
    }
    c->shadow = static_cast<float*>(p);
    if (c->p.storage == LBM3_REDUCED) {
      const cudaError_t e = lbm3::encode_population_maps(c->shadow_map, c->shadow, c->p.nx, c->p.ny, LBM3_FP32);
      if (e != cudaSuccess) return cuda_fail(c, e, "encoding the TMA descriptor of the FP32 shadow");
    }
  }
  *out = c->shadow;
  return LBM3_OK;
}

lbm3_status commit_fp32(lbm3_ctx* c) {
  if (c->p.storage == LBM3_FP32) return LBM3_OK;
  if (c->p.storage == LBM3_REDUCED) {
    c->in_shadow = true;
    return LBM3_OK;
  }
  LBM3_CUDA(c, lbm3::launch_encode(c->shadow, c->buf[c->cur], c->p.nx, c->p.ny, c->p.storage, c->stream));
  return LBM3_OK;
}

// The current state as a step's input: buffer, TMA descriptors and storage
// (the FP32 shadow while a reduced-storage state is still populations).
struct StateIn {
  const float* buf;
  const void* map;
  int storage;
};
StateIn state_in(const lbm3_ctx* c) {
  if (c->p.storage == LBM3_REDUCED && c->in_shadow) return {c->shadow, c->shadow_map, LBM3_FP32};
  return {c->buf[c->cur], c->tmap[c->cur], c->p.storage};
}

// FP32 stored populations of the current state: the current buffer (FP32
// storage) or the shadow, decoded (16-bit) or expanded (reduced) into it.
lbm3_status fp32_state(lbm3_ctx* c, const float** out) {
  if (c->p.storage == LBM3_FP32) {
    *out = c->buf[c->cur];
    return LBM3_OK;
  }
  float* sh = nullptr;
  lbm3_status st = fp32_target(c, &sh);
  if (st != LBM3_OK) return st;
  if (c->p.storage == LBM3_REDUCED) {
    if (!c->in_shadow)
      LBM3_CUDA(c, lbm3::launch_expand_reduced(c->buf[c->cur], sh, c->p.nx, c->p.ny, c->base, c->stream));
  } else {
    LBM3_CUDA(c, lbm3::launch_decode(c->buf[c->cur], sh, c->p.nx, c->p.ny, c->p.storage, c->stream));
  }
  *out = sh;
  return LBM3_OK;
}

// planes of FP64 data that fit in the staging buffer at once
int staging_planes(const lbm3_ctx* c) {
  const size_t per = nodes(c->p) * sizeof(double);
  size_t n = c->buf_bytes / per;
  return static_cast<int>(n > 13 ? 13 : (n < 1 ? 1 : n));
}

// Read and clear the device error word (synchronises the stream).
lbm3_status check_device_errors(lbm3_ctx* c) {
  LBM3_CUDA(c, cudaStreamSynchronize(c->stream));
  unsigned int e = 0;
  LBM3_CUDA(c, cudaMemcpy(&e, c->err, sizeof e, cudaMemcpyDeviceToHost));
  if (e) {
    LBM3_CUDA(c, cudaMemset(c->err, 0, sizeof e));
    return fail(c, LBM3_ETIMEOUT, "lbm3: a bounded wait inside the step kernel timed out (error word %u)", e);
  }
  return LBM3_OK;
}

// Row-chunk heights of the single-grid step kernel: H for the full-width
// strips and H_last for a narrower last strip, sized so that one wave of
// resident CTAs covers the grid.  The last strip's CTAs take the resident
// slots the full strips leave free; among the choices the one with the
// smallest estimated makespan max(H + 4, rho (H_last + 4)) wins, with rho the
// cost per row of the narrow strip relative to a full one (the work scales
// with its width, the per-row latency of the row pipeline does not).
constexpr double kNarrowRowBase = 0.5;  // rho = base + (1 - base) width / kTX

void tiling(const lbm3_ctx* c, StepArgs* a, int* grid) {
  const int nx = c->p.nx, ny = c->p.ny;
  const int nfs = nx / lbm3::kTX;
  const int wl = nx - nfs * lbm3::kTX;
  auto ceil_div = [](int x, int y) { return (x + y - 1) / y; };
  auto clamp_rows = [ny](int H) { return H < 4 ? (ny < 4 ? ny : 4) : (H > ny ? ny : H); };
  int H = c->rows_override, HL = c->rows_override;
  if (H <= 0) {
    const int resident = (c->occ > 0 ? c->occ : 1) * (c->num_sms > 0 ? c->num_sms : 1);
    const int nstrips = nfs + (wl > 0 ? 1 : 0);
    // small grids: short columns keep the pipeline fill short (H >= 4)
    H = HL = ceil_div(ny, resident / nstrips > 1 ? resident / nstrips : 1);
    if (wl > 0 && nfs > 0) {
      const double rho = kNarrowRowBase + (1.0 - kNarrowRowBase) * wl / lbm3::kTX;
      double best = 1e300;
      for (int cf = 1; nfs * cf < resident; ++cf) {
        const int h = ceil_div(ny, cf), hl = ceil_div(ny, resident - nfs * cf);
        const double t = std::max(h + 4.0, rho * (hl + 4.0));
        if (t < best) {
          best = t;
          H = h;
          HL = hl;
        }
        if (h <= 4) break;
      }
    }
  }
  H = clamp_rows(H);
  HL = clamp_rows(HL);
  a->rows_per_cta = H;
  a->rows_last = HL;
  a->full_blocks = nfs * ceil_div(ny, H);
  *grid = a->full_blocks + (wl > 0 ? ceil_div(ny, HL) : 0);
}

StepArgs args_for(const lbm3_ctx* c, const float* fin, float* fout, int* grid) {
  StepArgs a = c->base;
  a.fin = fin;
  a.fout = fout;
  if (c->p.storage == LBM3_FP16_DEV || c->p.storage == LBM3_BF16_DEV) {
    const size_t PS = static_cast<size_t>(lbm3::pitch_of(c->p.nx)) * c->p.ny;
    a.din = reinterpret_cast<const unsigned short*>(fin);
    a.dout = reinterpret_cast<unsigned short*>(fout);
    a.rin = fin ? reinterpret_cast<const float*>(a.din + 27 * PS) : nullptr;
    a.rout = fout ? reinterpret_cast<float*>(a.dout + 27 * PS) : nullptr;
  }
  tiling(c, &a, grid);
  return a;
}


// ------------------------------------------------------------ reverse mode
// d h_q / d sigma_r of the per-pair beta coefficients that fill_constants()
// derives from the tensions (h_q = g(X_q) for Eqs. 19-20; the sine terms of
// Eqs. 16 and 17), with X_q of Eq. 18.  Zero where h does not depend on sigma.
void beta_h_jacobian(const lbm3_params& p, double J[3][3]) {
  const double s[3] = {p.sigma12, p.sigma13, p.sigma23};
  const int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2};
  auto pidx = [](int k, int l) {
    const int lo = k < l ? k : l, hi = k < l ? l : k;
    return lo == 0 ? (hi == 1 ? 0 : 1) : 2;
  };
  double X[3], dX[3][3] = {{0.0}};
  bool tri = true;
  for (int q = 0; q < 3; ++q) {
    const int k = pk[q], l = pl[q], m = 3 - k - l;
    const int ia = pidx(m, k), ib = pidx(m, l), ic = pidx(k, l);
    const double a = s[ia], b = s[ib], c = s[ic];
    X[q] = (a * a + b * b - c * c) / (2.0 * a * b);
    dX[q][ia] = (a * a - b * b + c * c) / (2.0 * a * a * b);
    dX[q][ib] = (b * b - a * a + c * c) / (2.0 * a * b * b);
    dX[q][ic] = -c / (a * b);
    tri = tri && std::fabs(X[q]) < 1.0;
  }
  double dh_dX[3][3] = {{0.0}};  // dh_q / dX_r
  switch (p.beta_form) {
    case LBM3_BETA_PAPER:  // g(X) = -sgn(X)(1 - sqrt(1 - X^2)) inside [-1, 1]
      for (int q = 0; q < 3; ++q)
        if (std::fabs(X[q]) < 1.0) dh_dX[q][q] = -std::fabs(X[q]) / std::sqrt(1.0 - X[q] * X[q]);
      break;
    case LBM3_BETA_SPENCER:  // h_1 = sin(acos X_23) - 1, h_2 = sin(acos X_13) - 1
      if (tri) {
        dh_dX[1][2] = -X[2] / std::sqrt(1.0 - X[2] * X[2]);
        dh_dX[2][1] = -X[1] / std::sqrt(1.0 - X[1] * X[1]);
      }
      break;
    case LBM3_BETA_LECLAIRE:  // h_q = sin(a_m + a_q) - 1, a = acos X, m the largest angle
      if (tri) {
        double ang[3];
        for (int q = 0; q < 3; ++q) ang[q] = std::acos(X[q]);
        int qm = 0;
        for (int q = 1; q < 3; ++q)
          if (ang[q] > ang[qm]) qm = q;
        for (int q = 0; q < 3; ++q) {
          if (q == qm) continue;
          const double cq = std::cos(ang[qm] + ang[q]);
          dh_dX[q][q] += -cq / std::sqrt(1.0 - X[q] * X[q]);
          dh_dX[q][qm] += -cq / std::sqrt(1.0 - X[qm] * X[qm]);
        }
      }
      break;
    default:
      break;
  }
  for (int q = 0; q < 3; ++q)
    for (int r = 0; r < 3; ++r) {
      double v = 0.0;
      for (int j = 0; j < 3; ++j) v += dh_dX[q][j] * dX[j][r];
      J[q][r] = v;
    }
}

size_t slot_bytes(const lbm3_ctx* c) { return (c->buf_bytes + 255) / 256 * 256; }

float* slot(unsigned char* base, const lbm3_ctx* c, size_t i) {
  return reinterpret_cast<float*>(base + i * slot_bytes(c));
}

lbm3_status grow(lbm3_ctx* c, unsigned char** p, size_t* have, std::vector<unsigned char>* maps, size_t want,
                 const char* what) {
  if (*have >= want) return LBM3_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  maps->clear();
  if (want == 0) return LBM3_OK;
  void* q = nullptr;
  if (cudaMalloc(&q, want * slot_bytes(c)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LBM3_ENOMEM, "lbm3: cannot allocate %zu states (%zu bytes) for %s", want, want * slot_bytes(c),
                what);
  }
  *p = static_cast<unsigned char*>(q);
  *have = want;
  maps->assign(want * 256, 0);
  for (size_t i = 0; i < want; ++i) {
    const cudaError_t e =
        lbm3::encode_population_maps(maps->data() + i * 256, slot(*p, c, i), c->p.nx, c->p.ny, c->p.storage);
    if (e != cudaSuccess) return cuda_fail(c, e, "encoding the TMA descriptor of a tape state");
  }
  return LBM3_OK;
}

lbm3_status ensure_adjoint(lbm3_ctx* c) {
  if (c->adj) return LBM3_OK;
  const int N = static_cast<int>(nodes(c->p));
  void* a = nullptr;
  void* b = nullptr;
  if (cudaMalloc(&a, lbm3::adj_scratch_floats(N) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b, static_cast<size_t>(lbm3::adj_blocks(N)) * 6 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaFree(a);
    return fail(c, LBM3_ENOMEM, "lbm3: cannot allocate the reverse-mode scratch");
  }
  c->adj = static_cast<float*>(a);
  c->acc = static_cast<double*>(b);
  return LBM3_OK;
}

// one forward step from state `in` (TMA descriptors `map`) into `out`
lbm3_status step_into(lbm3_ctx* c, const float* in, const void* map, float* out) {
  int grid = 0;
  StepArgs a = args_for(c, in, out, &grid);
  LBM3_CUDA(c, lbm3::launch_step(a, map, grid, lbm3::MODE_STEP, c->p.storage, c->p.force_form, c->stream));
  return LBM3_OK;
}

// State S_t of the recorded run: a checkpoint (t a multiple of the
// checkpoint interval) or a recomputed state of the current segment.
struct TapeState {
  const float* p;
  const void* map;
};
TapeState tape_state(lbm3_ctx* c, int64_t t) {
  const int64_t K = c->tape_every;
  if (t % K == 0) {
    const size_t i = static_cast<size_t>(t / K);
    return {slot(c->ckpt, c, i), c->ckpt_maps.data() + i * 256};
  }
  const size_t j = static_cast<size_t>(t % K - 1);
  return {slot(c->tape, c, j), c->tape_maps.data() + j * 256};
}

// recompute the non-checkpoint states of segment r into the tape
lbm3_status recompute_segment(lbm3_ctx* c, int64_t r) {
  const int64_t K = c->tape_every, t0 = r * K;
  const int64_t end = (t0 + K < c->tape_steps) ? t0 + K : c->tape_steps;  // exclusive; S_end is not needed
  for (int64_t t = t0 + 1; t < end; ++t) {
    const TapeState in = tape_state(c, t - 1), out = tape_state(c, t);
    lbm3_status st = step_into(c, in.p, in.map, const_cast<float*>(out.p));
    if (st != LBM3_OK) return st;
  }
  return LBM3_OK;
}

}  // namespace

extern "C" {

lbm3_status lbm3_buffer_bytes(const lbm3_params* p, size_t* bytes) {
  std::string why;
  if (!bytes) return LBM3_EINVAL;
  lbm3_status st = validate(p, &why);
  if (st != LBM3_OK) return st;
  *bytes = buffer_bytes(*p);
  return LBM3_OK;
}

lbm3_status lbm3_create(const lbm3_params* p, void* cuda_stream, lbm3_ctx** out) {
  if (!out) return LBM3_EINVAL;
  *out = nullptr;
  std::string why;
  lbm3_status st = validate(p, &why);
  if (st != LBM3_OK) {
    std::fprintf(stderr, "%s\n", why.c_str());
    return st;
  }
  lbm3_ctx* c = new (std::nothrow) lbm3_ctx();
  if (!c) return LBM3_ENOMEM;
  c->p = *p;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->buf_bytes = buffer_bytes(*p);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = lbm3::step_configure();
  if (e == cudaSuccess) e = static_cast<cudaError_t>(lbm3::step_occupancy(&c->occ));
  if (e != cudaSuccess) {
    std::fprintf(stderr, "lbm3_create: %s\n", cudaGetErrorString(e));
    delete c;
    return LBM3_ECUDA;
  }
  c->red_blocks = lbm3::reduce_blocks(static_cast<int>(nodes(*p)));
  const size_t scratch_bytes = static_cast<size_t>(c->red_blocks) * 5 * sizeof(double) + 8 * sizeof(double) + 256;
  void* sp = nullptr;
  if (cudaMalloc(&sp, scratch_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return LBM3_ENOMEM;
  }
  c->scratch = static_cast<unsigned char*>(sp);
  c->partial = reinterpret_cast<double*>(c->scratch);
  c->red_out = c->partial + static_cast<size_t>(c->red_blocks) * 5;
  c->err = reinterpret_cast<unsigned int*>(c->red_out + 5);
  c->bad = c->err + 1;
  if (cudaMemset(c->scratch, 0, scratch_bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sp);
    delete c;
    return LBM3_ECUDA;
  }
  StepArgs& a = c->base;
  a.nx = p->nx;
  a.ny = p->ny;
  a.pitch = lbm3::pitch_of(p->nx);
  a.boxw = lbm3::kPW;  // pitch_of() is never below one box
  a.nstrips = (p->nx + lbm3::kTX - 1) / lbm3::kTX;
  a.err = c->err;
  a.stall_row = -1;
  fill_constants(*p, &a);
  *out = c;
  return LBM3_OK;
}

lbm3_status lbm3_bind_buffers(lbm3_ctx* c, void* f0, void* f1, size_t bytes_each) {
  if (!c) return LBM3_EINVAL;
  if (c->state_set || c->buf[0]) return fail(c, LBM3_ESTATE, "lbm3_bind_buffers: buffers already set");
  if (!f0 || !f1 || f0 == f1) return fail(c, LBM3_EINVAL, "lbm3_bind_buffers: need two distinct buffers");
  if (bytes_each < c->buf_bytes)
    return fail(c, LBM3_EINVAL, "lbm3_bind_buffers: %zu bytes < required %zu", bytes_each, c->buf_bytes);
  if ((reinterpret_cast<uintptr_t>(f0) | reinterpret_cast<uintptr_t>(f1)) & 255u)
    return fail(c, LBM3_EINVAL, "lbm3_bind_buffers: buffers must be 256-byte aligned");
  c->buf[0] = static_cast<float*>(f0);
  c->buf[1] = static_cast<float*>(f1);
  c->owns_bufs = false;
  DeviceGuard g(c->device);
  return encode_maps(c);
}

lbm3_status lbm3_init(lbm3_ctx* c, const double* rho, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!rho) return fail(c, LBM3_EINVAL, "lbm3_init: NULL rho");
  DeviceGuard g(c->device);
  lbm3_status st = ensure_buffers(c);
  if (st != LBM3_OK) return st;
  const size_t N = nodes(c->p);
  const double* src = rho;
  if (!on_device) {
    for (size_t n = 0; n < N; ++n) {
      const double a = rho[n], b = rho[N + n], d = rho[2 * N + n];
      if (!(std::isfinite(a) && std::isfinite(b) && std::isfinite(d) && a >= 0.0 && b >= 0.0 && d >= 0.0 &&
            a + b + d > 0.0))
        return fail(c, LBM3_EINVAL, "lbm3_init: rho at node %zu is invalid (needs rho_k >= 0, sum > 0)", n);
    }
    double* staging = reinterpret_cast<double*>(c->buf[c->cur ^ 1]);
    LBM3_CUDA(c, cudaMemcpyAsync(staging, rho, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    src = staging;
  } else {
    LBM3_CUDA(c, cudaMemsetAsync(c->bad, 0, sizeof(unsigned int), c->stream));
    LBM3_CUDA(c, lbm3::launch_check_rho(rho, static_cast<int>(N), c->bad, c->stream));
    unsigned int bad = 0;
    LBM3_CUDA(c, cudaMemcpyAsync(&bad, c->bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
    LBM3_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, LBM3_EINVAL, "lbm3_init: device rho has a node with rho_k < 0, NaN or sum 0");
  }
  float* target = nullptr;
  st = fp32_target(c, &target);
  if (st != LBM3_OK) return st;
  LBM3_CUDA(c, lbm3::launch_init_from_rho(src, target, c->p.nx, c->p.ny, c->stream));
  st = commit_fp32(c);
  if (st != LBM3_OK) return st;
  if (!on_device) LBM3_CUDA(c, cudaStreamSynchronize(c->stream));  // staging reused next
  c->state_set = true;
  c->tape_valid = false;
  c->t = 0;
  return LBM3_OK;
}

lbm3_status lbm3_set_populations(lbm3_ctx* c, const double* f, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!f) return fail(c, LBM3_EINVAL, "lbm3_set_populations: NULL f");
  DeviceGuard g(c->device);
  lbm3_status st = ensure_buffers(c);
  if (st != LBM3_OK) return st;
  const size_t N = nodes(c->p);
  float* target = nullptr;
  st = fp32_target(c, &target);
  if (st != LBM3_OK) return st;
  if (on_device) {
    LBM3_CUDA(c, lbm3::launch_set_planes(f, target, c->p.nx, c->p.ny, 0, 27, c->stream));
  } else {
    double* staging = reinterpret_cast<double*>(c->buf[c->cur ^ 1]);
    const int chunk = staging_planes(c);
    for (int p0 = 0; p0 < 27; p0 += chunk) {
      const int np = p0 + chunk <= 27 ? chunk : 27 - p0;
      LBM3_CUDA(c, cudaMemcpyAsync(staging, f + static_cast<size_t>(p0) * N, np * N * sizeof(double),
                                   cudaMemcpyHostToDevice, c->stream));
      LBM3_CUDA(c, lbm3::launch_set_planes(staging, target, c->p.nx, c->p.ny, p0, np, c->stream));
      LBM3_CUDA(c, cudaStreamSynchronize(c->stream));
    }
  }
  st = commit_fp32(c);
  if (st != LBM3_OK) return st;
  c->state_set = true;
  c->tape_valid = false;
  c->t = 0;
  return LBM3_OK;
}

lbm3_status lbm3_set_rows_per_cta(lbm3_ctx* c, int32_t rows) {
  if (!c) return LBM3_EINVAL;
  if (rows < 0 || rows > c->p.ny) return fail(c, LBM3_EINVAL, "lbm3_set_rows_per_cta: %d not in [0, ny]", rows);
  c->rows_override = rows;
  return LBM3_OK;
}

lbm3_status lbm3_debug_stall_row(lbm3_ctx* c, int32_t row) {
  if (!c) return LBM3_EINVAL;
  if (row < -1) return fail(c, LBM3_EINVAL, "lbm3_debug_stall_row: row %d < -1", row);
  c->stall_row = row;
  return LBM3_OK;
}

lbm3_status lbm3_step(lbm3_ctx* c, int64_t n) {
  if (!c) return LBM3_EINVAL;
  if (n < 0) return fail(c, LBM3_EINVAL, "lbm3_step: n = %lld < 0", static_cast<long long>(n));
  if (!c->state_set) return fail(c, LBM3_ESTATE, "lbm3_step: state not initialised");
  DeviceGuard g(c->device);
  if (n > 0) c->tape_valid = false;
  for (int64_t s = 0; s < n; ++s) {
    int grid = 0;
    const StateIn in = state_in(c);
    // a reduced-storage state that is still populations: FP32 in, reduced out
    const int storage = in.storage == c->p.storage ? c->p.storage : lbm3::ST_F2R;
    StepArgs a = args_for(c, in.buf, c->buf[c->cur ^ 1], &grid);
    a.stall_row = c->stall_row;
    c->stall_row = -1;
    LBM3_CUDA(c, lbm3::launch_step(a, in.map, grid, lbm3::MODE_STEP, storage, c->p.force_form, c->stream));
    c->cur ^= 1;
    c->in_shadow = false;
    c->t += 1;
  }
  return LBM3_OK;
}

lbm3_status lbm3_fields(lbm3_ctx* c, double* rho, double* ux, double* uy, double* pr, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!c->state_set) return fail(c, LBM3_ESTATE, "lbm3_fields: state not initialised");
  DeviceGuard g(c->device);
  const size_t N = nodes(c->p);
  int grid = 0;
  const StateIn in = state_in(c);
  StepArgs a = args_for(c, in.buf, nullptr, &grid);
  double* staging = reinterpret_cast<double*>(c->buf[c->cur ^ 1]);
  if (on_device) {
    a.out_rho = rho;
    a.out_ux = ux;
    a.out_uy = uy;
    a.out_p = pr;
  } else {
    a.out_rho = rho ? staging : nullptr;
    a.out_ux = ux ? staging + 3 * N : nullptr;
    a.out_uy = uy ? staging + 4 * N : nullptr;
    a.out_p = pr ? staging + 5 * N : nullptr;
  }
  LBM3_CUDA(c, lbm3::launch_step(a, in.map, grid, lbm3::MODE_FIELDS, in.storage, c->p.force_form, c->stream));
  if (!on_device) {
    if (rho) LBM3_CUDA(c, cudaMemcpyAsync(rho, staging, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (ux) LBM3_CUDA(c, cudaMemcpyAsync(ux, staging + 3 * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (uy) LBM3_CUDA(c, cudaMemcpyAsync(uy, staging + 4 * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (pr) LBM3_CUDA(c, cudaMemcpyAsync(pr, staging + 5 * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return check_device_errors(c);
  }
  return LBM3_OK;
}

lbm3_status lbm3_populations(lbm3_ctx* c, double* f, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!f) return fail(c, LBM3_EINVAL, "lbm3_populations: NULL f");
  if (!c->state_set) return fail(c, LBM3_ESTATE, "lbm3_populations: state not initialised");
  DeviceGuard g(c->device);
  const size_t N = nodes(c->p);
  const float* src = nullptr;
  lbm3_status st0 = fp32_state(c, &src);
  if (st0 != LBM3_OK) return st0;
  if (on_device) {
    LBM3_CUDA(c, lbm3::launch_get_planes(src, f, c->p.nx, c->p.ny, 0, 27, c->stream));
    return LBM3_OK;
  }
  double* staging = reinterpret_cast<double*>(c->buf[c->cur ^ 1]);
  const int chunk = staging_planes(c);
  for (int p0 = 0; p0 < 27; p0 += chunk) {
    const int np = p0 + chunk <= 27 ? chunk : 27 - p0;
    LBM3_CUDA(c, lbm3::launch_get_planes(src, staging, c->p.nx, c->p.ny, p0, np, c->stream));
    LBM3_CUDA(c, cudaMemcpyAsync(f + static_cast<size_t>(p0) * N, staging, np * N * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
    LBM3_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return check_device_errors(c);
}

lbm3_status lbm3_mass(lbm3_ctx* c, double* mass, double* mom) {
  if (!c) return LBM3_EINVAL;
  if (!c->state_set) return fail(c, LBM3_ESTATE, "lbm3_mass: state not initialised");
  DeviceGuard g(c->device);
  if (c->p.storage == LBM3_FP32 || c->p.storage == LBM3_REDUCED) {
    const float* src = nullptr;
    lbm3_status st0 = fp32_state(c, &src);
    if (st0 != LBM3_OK) return st0;
    LBM3_CUDA(c, lbm3::launch_reduce_padded(src, c->p.nx, c->p.ny, c->partial, c->red_blocks, c->red_out,
                                            c->stream));
  } else
    LBM3_CUDA(c, lbm3::launch_reduce_dev(c->buf[c->cur], c->p.nx, c->p.ny, c->p.storage, c->partial,
                                         c->red_blocks, c->red_out, c->stream));
  double h[5];
  LBM3_CUDA(c, cudaMemcpyAsync(h, c->red_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  lbm3_status st = check_device_errors(c);
  if (st != LBM3_OK) return st;
  if (mass)
    for (int k = 0; k < 3; ++k) mass[k] = h[k];
  if (mom) {
    mom[0] = h[3];
    mom[1] = h[4];
  }
  for (int j = 0; j < 5; ++j)
    if (!std::isfinite(h[j])) return fail(c, LBM3_ENUMERIC, "lbm3_mass: non-finite sum (NaN/Inf in the state)");
  return LBM3_OK;
}

lbm3_status lbm3_interface_diagnostics(lbm3_ctx* c, double third_max, double bulk_min, lbm3_interfaces* out) {
  if (!c) return LBM3_EINVAL;
  if (!out) return fail(c, LBM3_EINVAL, "lbm3_interface_diagnostics: NULL out");
  if (!(third_max > 0.0 && third_max <= 1.0) || !(bulk_min > 0.0 && bulk_min < 1.0))
    return fail(c, LBM3_EINVAL, "lbm3_interface_diagnostics: need 0 < third_max <= 1 and 0 < bulk_min < 1");
  if (!c->state_set) return fail(c, LBM3_ESTATE, "lbm3_interface_diagnostics: state not initialised");
  DeviceGuard g(c->device);
  if (!c->diag) {
    void* q = nullptr;
    if (cudaMalloc(&q, lbm3::diag_scratch_doubles() * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, LBM3_ENOMEM, "lbm3_interface_diagnostics: cannot allocate the diagnostic scratch");
    }
    c->diag = static_cast<double*>(q);
  }
  const size_t N = nodes(c->p);
  int grid = 0;
  const StateIn in = state_in(c);
  StepArgs a = args_for(c, in.buf, nullptr, &grid);
  // FP64 rho_k and p of the current state in the idle buffer (32 bytes per node)
  double* staging = reinterpret_cast<double*>(c->buf[c->cur ^ 1]);
  a.out_rho = staging;
  a.out_p = staging + 3 * N;
  LBM3_CUDA(c, lbm3::launch_step(a, in.map, grid, lbm3::MODE_FIELDS, in.storage, c->p.force_form, c->stream));
  LBM3_CUDA(c, lbm3::launch_diag(staging, staging + 3 * N, c->p.nx, c->p.ny, third_max, bulk_min, c->diag,
                                 c->stream));
  double sums[33];
  LBM3_CUDA(c, cudaMemcpyAsync(sums, c->diag + static_cast<size_t>(lbm3::kDiagMaxBlocks) * 33, sizeof sums,
                               cudaMemcpyDeviceToHost, c->stream));
  lbm3_status st = check_device_errors(c);
  if (st != LBM3_OK) return st;
  lbm3::diag_geometry(sums, c->p.nx, c->p.ny, out);
  return LBM3_OK;
}

lbm3_status lbm3_sync(lbm3_ctx* c) {
  if (!c) return LBM3_EINVAL;
  DeviceGuard g(c->device);
  return check_device_errors(c);
}

int64_t lbm3_time(const lbm3_ctx* c) { return c ? c->t : -1; }

lbm3_status lbm3_destroy(lbm3_ctx* c) {
  if (!c) return LBM3_OK;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->owns_bufs) {
    cudaFree(c->buf[0]);
    cudaFree(c->buf[1]);
  }
  if (c->shadow) cudaFree(c->shadow);
  if (c->diag) cudaFree(c->diag);
  if (c->ckpt) cudaFree(c->ckpt);
  if (c->tape) cudaFree(c->tape);
  if (c->adj) cudaFree(c->adj);
  if (c->acc) cudaFree(c->acc);
  cudaFree(c->scratch);
  cudaGetLastError();
  delete c;
  return LBM3_OK;
}


lbm3_status lbm3_set_params(lbm3_ctx* c, const lbm3_params* p) {
  if (!c) return LBM3_EINVAL;
  std::string why;
  if (validate(p, &why) != LBM3_OK) return fail(c, LBM3_EINVAL, "%s", why.c_str());
  if (p->nx != c->p.nx || p->ny != c->p.ny || p->storage != c->p.storage)
    return fail(c, LBM3_EINVAL, "lbm3_set_params: nx, ny and storage cannot change");
  if (c->p.storage == LBM3_REDUCED && c->state_set && !c->in_shadow) {
    // the reduced state's populations are formed with the recolouring
    // weights of the step that produced them: expand them with those weights
    const float* sh = nullptr;
    lbm3_status st = fp32_state(c, &sh);
    if (st != LBM3_OK) return st;
    c->in_shadow = true;
  }
  c->p = *p;
  fill_constants(*p, &c->base);
  c->tape_valid = false;
  return LBM3_OK;
}

lbm3_status lbm3_phi(lbm3_ctx* c, double* phi, int on_device) {
  if (!c) return LBM3_EINVAL;
  if (!phi) return fail(c, LBM3_EINVAL, "lbm3_phi: NULL phi");
  if (!c->state_set) return fail(c, LBM3_ESTATE, "lbm3_phi: state not initialised");
  if (c->p.storage != LBM3_FP32 && c->p.storage != LBM3_REDUCED)
    return fail(c, LBM3_EINVAL, "lbm3_phi: needs FP32 or reduced storage (use lbm3_fields)");
  DeviceGuard g(c->device);
  const size_t N = nodes(c->p);
  const float* src = nullptr;
  lbm3_status st0 = fp32_state(c, &src);
  if (st0 != LBM3_OK) return st0;
  double* dst = on_device ? phi : reinterpret_cast<double*>(c->buf[c->cur ^ 1]);
  LBM3_CUDA(c, lbm3::launch_phi(src, dst, c->p.nx, c->p.ny, c->stream));
  if (on_device) return LBM3_OK;
  LBM3_CUDA(c, cudaMemcpyAsync(phi, dst, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check_device_errors(c);
}

lbm3_status lbm3_tape_forward(lbm3_ctx* c, int64_t nsteps, int32_t every) {
  if (!c) return LBM3_EINVAL;
  if (nsteps < 1 || every < 1)
    return fail(c, LBM3_EINVAL, "lbm3_tape_forward: nsteps = %lld and checkpoint_every = %d must be >= 1",
                static_cast<long long>(nsteps), every);
  if (!c->state_set) return fail(c, LBM3_ESTATE, "lbm3_tape_forward: state not initialised");
  if (c->p.storage != LBM3_FP32 || c->p.force_form != LBM3_FORCE_BODY)
    return fail(c, LBM3_EINVAL, "lbm3_tape_forward: reverse mode needs FP32 storage and the body force form");
  DeviceGuard g(c->device);
  c->tape_valid = false;
  const size_t nseg = static_cast<size_t>((nsteps + every - 1) / every);
  const size_t seg = static_cast<size_t>(nsteps < every ? nsteps : every);
  lbm3_status st = grow(c, &c->ckpt, &c->ckpt_slots, &c->ckpt_maps, nseg, "checkpoints");
  if (st == LBM3_OK) st = grow(c, &c->tape, &c->tape_slots, &c->tape_maps, seg - 1, "the segment tape");
  if (st == LBM3_OK) st = ensure_adjoint(c);
  if (st != LBM3_OK) return st;
  c->tape_every = every;
  c->tape_steps = nsteps;
  // S_0 into its checkpoint; each later checkpoint is written by the step
  // that produces it, other states ping-pong through the context's buffers
  LBM3_CUDA(c, cudaMemcpyAsync(slot(c->ckpt, c, 0), c->buf[c->cur], c->buf_bytes, cudaMemcpyDeviceToDevice,
                               c->stream));
  TapeState cur = tape_state(c, 0);
  for (int64_t t = 1; t <= nsteps; ++t) {
    const bool keep = (t % every == 0) && t < nsteps;
    float* out = keep ? const_cast<float*>(tape_state(c, t).p) : (cur.p == c->buf[0] ? c->buf[1] : c->buf[0]);
    st = step_into(c, cur.p, cur.map, out);
    if (st != LBM3_OK) return st;
    if (keep) {
      cur = tape_state(c, t);
    } else {
      const int b = out == c->buf[0] ? 0 : 1;
      cur = {c->buf[b], c->tmap[b]};
    }
    c->t += 1;
  }
  c->cur = cur.p == c->buf[0] ? 0 : 1;  // S_nsteps is in a context buffer
  c->tape_valid = true;
  return LBM3_OK;
}

lbm3_status lbm3_tape_backward(lbm3_ctx* c, const double* dphi, int dphi_on_device, double* dpop0, double* drho0,
                               int out_on_device, double* dsigma) {
  if (!c) return LBM3_EINVAL;
  if (!dphi) return fail(c, LBM3_EINVAL, "lbm3_tape_backward: NULL dphi");
  if (!c->tape_valid) return fail(c, LBM3_ESTATE, "lbm3_tape_backward: no recorded run (lbm3_tape_forward)");
  DeviceGuard g(c->device);
  const int nx = c->p.nx, ny = c->p.ny, N = nx * ny;
  lbm3::AdjBuffers b;
  lbm3::adj_layout(c->adj, N, &b);
  const int nblk = lbm3::adj_blocks(N);
  LBM3_CUDA(c, cudaMemsetAsync(c->acc, 0, static_cast<size_t>(nblk) * 6 * sizeof(double), c->stream));
  const double* dphi_d = dphi;
  if (!dphi_on_device) {  // staged in the second lam9 buffer, free until the first adjoint step
    double* stage = reinterpret_cast<double*>(b.lam9[1]);
    LBM3_CUDA(c, cudaMemcpyAsync(stage, dphi, 3 * static_cast<size_t>(N) * sizeof(double), cudaMemcpyHostToDevice,
                                 c->stream));
    dphi_d = stage;
  }
  LBM3_CUDA(c, lbm3::launch_adj_seed(c->buf[c->cur], dphi_d, b, 0, nx, ny, c->stream));
  const int64_t T = c->tape_steps, K = c->tape_every;
  int grid = 0;
  const StepArgs a = args_for(c, nullptr, nullptr, &grid);
  int64_t seg = (T - 1) / K;  // segment whose states are in the tape
  lbm3_status st = recompute_segment(c, seg);
  if (st != LBM3_OK) return st;
  LBM3_CUDA(c, lbm3::launch_adj_fields(tape_state(c, T - 1).p, a, b, 0, c->stream));
  int slotf = 0, lam = 0;
  for (int64_t t = T; t >= 1; --t) {
    const float* prev = tape_state(c, t - 1).p;
    const float* next = nullptr;
    if (t >= 2) {
      if ((t - 2) / K != seg) {  // S_{t-1} is a checkpoint: the tape is free to refill
        seg = (t - 2) / K;
        st = recompute_segment(c, seg);
        if (st != LBM3_OK) return st;
      }
      next = tape_state(c, t - 2).p;
    }
    LBM3_CUDA(c, lbm3::launch_adj_step(prev, next, a, b, slotf, lam, c->acc, c->stream));
    slotf ^= 1;
    lam ^= 1;
  }
  double* staging = reinterpret_cast<double*>(c->buf[c->cur ^ 1]);
  if (dpop0) {
    if (out_on_device) {
      LBM3_CUDA(c, lbm3::launch_adj_dpop(b, lam, dpop0, nx, ny, 0, 27, c->stream));
    } else {
      const int chunk = staging_planes(c);
      for (int p0 = 0; p0 < 27; p0 += chunk) {
        const int np = p0 + chunk <= 27 ? chunk : 27 - p0;
        LBM3_CUDA(c, lbm3::launch_adj_dpop(b, lam, staging, nx, ny, p0, np, c->stream));
        LBM3_CUDA(c, cudaMemcpyAsync(dpop0 + static_cast<size_t>(p0) * N, staging,
                                     static_cast<size_t>(np) * N * sizeof(double), cudaMemcpyDeviceToHost,
                                     c->stream));
        LBM3_CUDA(c, cudaStreamSynchronize(c->stream));
      }
    }
  }
  if (drho0) {
    double* dst = out_on_device ? drho0 : staging;
    LBM3_CUDA(c, lbm3::launch_adj_drho(b, lam, dst, nx, ny, c->stream));
    if (!out_on_device)
      LBM3_CUDA(c, cudaMemcpyAsync(drho0, dst, 3 * static_cast<size_t>(N) * sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
  }
  std::vector<double> rows(static_cast<size_t>(nblk) * 6);
  LBM3_CUDA(c, cudaMemcpyAsync(rows.data(), c->acc, rows.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  st = check_device_errors(c);
  if (st != LBM3_OK) return st;
  double tot[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int r = 0; r < nblk; ++r)
    for (int j = 0; j < 6; ++j) tot[j] += rows[static_cast<size_t>(r) * 6 + j];
  for (int j = 0; j < 6; ++j)
    if (!std::isfinite(tot[j])) return fail(c, LBM3_ENUMERIC, "lbm3_tape_backward: non-finite gradient");
  if (dsigma) {
    double J[3][3];
    beta_h_jacobian(c->p, J);
    for (int r = 0; r < 3; ++r) {
      double v = tot[r];
      for (int q = 0; q < 3; ++q) v += tot[3 + q] * J[q][r];
      dsigma[r] = v;
    }
  }
  return LBM3_OK;
}

const char* lbm3_last_error(const lbm3_ctx* c) { return c ? c->msg.c_str() : kNullCtxMsg; }

}  // extern "C"

// ---------------------------------------------------------------- batches
// A batch is a set of independent simulations (own grid size and
// parameters) advanced together: one launch per step covers every tile of
// every instance, and steps are replayed from a captured two-step CUDA graph.
// Each instance is an ordinary context underneath, so per-instance set-up and
// read-out use the single-instance code paths.

struct lbm3_batch {
  std::vector<lbm3_ctx*> ctx;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  lbm3::BatchItem* d_items = nullptr;
  lbm3::BatchDesc* d_descs = nullptr;
  // per parity, the instances' step arguments for the kernel parameter space
  // (empty for batches of more than kBatchParamInst instances)
  std::vector<lbm3::BatchArgsBlock> pargs;
  int nitems = 0;
  size_t items_cap = 0;  // BatchItem slots allocated at d_items
  std::vector<lbm3::BatchItem> items;  // host copy of the work list
  lbm3::BatchItem* d_items2 = nullptr;  // reduced state: work lists of a split first step
  int storage = LBM3_FP32;
  int rows = 64;
  std::vector<int> ranked;  // tile heights ranked by the makespan model, best first
  int device = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // two steps, by starting parity
  int64_t t = 0;
  std::string msg;
};

namespace {

const char* kNullBatchMsg = "lbm3: NULL batch";

lbm3_status bfail(lbm3_batch* b, lbm3_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->msg = buf;
  return st;
}

lbm3_status bcheck(lbm3_batch* b, lbm3_status st, int i) {
  if (st != LBM3_OK && b) b->msg = std::string("instance ") + std::to_string(i) + ": " + b->ctx[i]->msg;
  return st;
}

void destroy_batch(lbm3_batch* b) {
  for (int p = 0; p < 2; ++p)
    if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
  for (lbm3_ctx* c : b->ctx) lbm3_destroy(c);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_items2) cudaFree(b->d_items2);
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaGetLastError();
  delete b;
}

const lbm3::BatchArgsBlock* param_args(const lbm3_batch* b, int parity) {
  return b->pargs.empty() ? nullptr : &b->pargs[static_cast<size_t>(parity)];
}

lbm3_status launch_one(lbm3_batch* b, int parity, cudaStream_t st) {
  const cudaError_t e =
      lbm3::launch_batch(b->d_items, b->nitems, b->d_descs, param_args(b, parity), parity, b->storage, st);
  if (e != cudaSuccess) return bfail(b, LBM3_ECUDA, "lbm3_batch_step: %s", cudaGetErrorString(e));
  return LBM3_OK;
}

lbm3_status build_graph(lbm3_batch* b, int parity) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = lbm3::launch_batch(b->d_items, b->nitems, b->d_descs, param_args(b, parity), parity,
                                        b->storage, b->cap_stream);
    cudaError_t e2 = lbm3::launch_batch(b->d_items, b->nitems, b->d_descs, param_args(b, parity ^ 1), parity ^ 1,
                                        b->storage, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
    if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[parity], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, LBM3_ECUDA, "lbm3_batch_step: graph capture failed: %s", cudaGetErrorString(e));
  }
  return LBM3_OK;
}

// Work items of every instance for tile height `rows` (equal-width strips of
// at most kTX columns, row chunks of `rows`), largest first.
void batch_items(const lbm3_batch* b, int rows, std::vector<lbm3::BatchItem>* out_items) {
  out_items->clear();
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const lbm3_ctx* c = b->ctx[i];
    const int ns = (c->p.nx + lbm3::kTX - 1) / lbm3::kTX;
    const int H = std::min(rows, c->p.ny);
    for (int y0 = 0; y0 < c->p.ny; y0 += H)
      for (int s = 0; s < ns; ++s) {
        const int x0 = lbm3::strip_x0(s, ns, c->p.nx);
        out_items->push_back(
            {static_cast<int>(i), x0, lbm3::strip_x0(s + 1, ns, c->p.nx) - x0, y0, std::min(H, c->p.ny - y0)});
      }
  }
  std::stable_sort(out_items->begin(), out_items->end(), [](const lbm3::BatchItem& a, const lbm3::BatchItem& c) {
    return a.w * (a.h + 4) > c.w * (c.h + 4);
  });
}

// Estimated step time of a work list: largest-first assignment of the items
// to the resident CTA slots, item cost ~ (h + 4 halo rows) x (w + 32 columns
// of per-row overhead).
double batch_makespan(const lbm3_batch* b, const std::vector<lbm3::BatchItem>& its) {
  const int slots = std::max(1, b->ctx[0]->occ * b->ctx[0]->num_sms);
  std::vector<double> load(static_cast<size_t>(slots), 0.0);
  for (const lbm3::BatchItem& it : its) {
    auto m = std::min_element(load.begin(), load.end());
    *m += static_cast<double>(it.h + 4) * (it.w + 32);
  }
  return *std::max_element(load.begin(), load.end());
}

// Upload a work list (growing the device array when needed).
lbm3_status batch_upload(lbm3_batch* b, const std::vector<lbm3::BatchItem>& items) {
  if (b->d_items) {  // launches in flight may still read the current list
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM3_ECUDA, "lbm3: batch work list: %s", cudaGetErrorString(e));
  }
  if (items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    if (cudaMalloc(&b->d_items, sizeof(lbm3::BatchItem) * items.size()) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, LBM3_ENOMEM, "lbm3: cannot allocate the batch work list");
    }
    b->items_cap = items.size();
  }
  const cudaError_t e =
      cudaMemcpy(b->d_items, items.data(), sizeof(lbm3::BatchItem) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bfail(b, LBM3_ECUDA, "lbm3: batch work list upload: %s", cudaGetErrorString(e));
  b->nitems = static_cast<int>(items.size());
  b->items = items;
  return LBM3_OK;
}

// Reduced state: the first step of instances whose state is still FP32
// populations (set since the last step) reads them and writes the reduced
// state; the other instances take an ordinary reduced step in a second
// launch of the same step.
lbm3_status batch_first_reduced_step(lbm3_batch* b, int parity) {
  std::vector<char> pop(b->ctx.size());
  size_t npop = 0;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    pop[i] = b->ctx[i]->in_shadow ? 1 : 0;
    npop += pop[i];
  }
  if (npop == 0) return LBM3_OK;
  cudaError_t e;
  if (npop == b->ctx.size()) {
    e = lbm3::launch_batch(b->d_items, b->nitems, b->d_descs, nullptr, parity, lbm3::ST_F2R, b->stream);
  } else {
    std::vector<lbm3::BatchItem> split;
    for (const lbm3::BatchItem& it : b->items)
      if (pop[static_cast<size_t>(it.inst)]) split.push_back(it);
    const int nf = static_cast<int>(split.size());
    for (const lbm3::BatchItem& it : b->items)
      if (!pop[static_cast<size_t>(it.inst)]) split.push_back(it);
    e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && !b->d_items2) e = cudaMalloc(&b->d_items2, sizeof(lbm3::BatchItem) * b->items_cap);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_items2, split.data(), sizeof(lbm3::BatchItem) * split.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = lbm3::launch_batch(b->d_items2, nf, b->d_descs, nullptr, parity, lbm3::ST_F2R, b->stream);
    if (e == cudaSuccess)
      e = lbm3::launch_batch(b->d_items2 + nf, static_cast<int>(split.size()) - nf, b->d_descs, param_args(b, parity),
                             parity, lbm3::ST_RED, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // d_items2 is rewritten by the next split
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, LBM3_ECUDA, "lbm3_batch_step: %s", cudaGetErrorString(e));
  }
  for (lbm3_ctx* c : b->ctx) c->in_shadow = false;
  return LBM3_OK;
}

}  // namespace

extern "C" {

lbm3_status lbm3_batch_create(const lbm3_params* params, int32_t count, void* cuda_stream, int32_t rows_per_cta,
                              lbm3_batch** out) {
  if (!out) return LBM3_EINVAL;
  *out = nullptr;
  if (!params || count <= 0 || rows_per_cta < 0) return LBM3_EINVAL;
  lbm3_batch* b = new (std::nothrow) lbm3_batch();
  if (!b) return LBM3_ENOMEM;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (rows_per_cta > 0) b->rows = rows_per_cta;
  cudaGetDevice(&b->device);
  for (int i = 0; i < count; ++i) {
    lbm3_ctx* c = nullptr;
    lbm3_status st = lbm3_create(&params[i], cuda_stream, &c);
    if (st != LBM3_OK) {
      std::fprintf(stderr, "lbm3_batch_create: instance %d rejected\n", i);
      destroy_batch(b);
      return st;
    }
    b->ctx.push_back(c);
    if ((c->p.storage != LBM3_FP32 && c->p.storage != LBM3_REDUCED) || c->p.storage != params[0].storage ||
        c->p.force_form != LBM3_FORCE_BODY) {
      std::fprintf(stderr,
                   "lbm3_batch_create: instance %d: batches use the body force and one storage for every instance, "
                   "FP32 or the reduced state\n",
                   i);
      destroy_batch(b);
      return LBM3_EINVAL;
    }
    st = ensure_buffers(c);
    if (st == LBM3_OK && c->p.storage == LBM3_REDUCED) {
      float* sh = nullptr;  // the FP32 populations a state is set to, and their descriptors
      st = fp32_target(c, &sh);
    }
    if (st != LBM3_OK) {
      std::fprintf(stderr, "lbm3_batch_create: instance %d: %s\n", i, c->msg.c_str());
      destroy_batch(b);
      return st;
    }
  }
  // per-instance descriptors and the work list (largest tiles first)
  std::vector<lbm3::BatchDesc> descs(count);
  std::vector<lbm3::BatchItem> items;
  b->storage = params[0].storage;
  for (int i = 0; i < count; ++i) {
    lbm3_ctx* c = b->ctx[i];
    for (int p = 0; p < 2; ++p) {
      int grid = 0;
      descs[i].args[p] = args_for(c, c->buf[p], c->buf[p ^ 1], &grid);
      std::memcpy(descs[i].map[p], c->tmap[p], 256);
      if (b->storage == LBM3_REDUCED) descs[i].args_f2r[p] = args_for(c, c->shadow, c->buf[p ^ 1], &grid);
    }
    if (b->storage == LBM3_REDUCED) std::memcpy(descs[i].map_f2r, c->shadow_map, 256);
  }
  // Tile height: given, or the one whose largest-first assignment of the work
  // items to the resident CTA slots gives the shortest estimated step.  The
  // heights are kept ranked by that estimate for lbm3_batch_autotune.
  {
    std::vector<std::pair<double, int>> est;
    for (int rows = 16; rows <= 512; rows += 8) {
      std::vector<lbm3::BatchItem> cand;
      batch_items(b, rows, &cand);
      est.push_back({batch_makespan(b, cand), rows});
    }
    std::stable_sort(est.begin(), est.end(),
                     [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x.first < y.first; });
    for (const auto& e : est) b->ranked.push_back(e.second);
  }
  if (rows_per_cta <= 0) b->rows = b->ranked[0];
  batch_items(b, b->rows, &items);
  if (count <= lbm3::kBatchParamInst) {
    b->pargs.assign(2, lbm3::BatchArgsBlock{});
    for (int p = 0; p < 2; ++p)
      for (int i = 0; i < count; ++i) b->pargs[static_cast<size_t>(p)].a[i] = descs[static_cast<size_t>(i)].args[p];
  }
  if (batch_upload(b, items) != LBM3_OK) {
    std::fprintf(stderr, "lbm3_batch_create: %s\n", b->msg.c_str());
    destroy_batch(b);
    return LBM3_ENOMEM;
  }
  cudaError_t e = cudaMalloc(&b->d_descs, sizeof(lbm3::BatchDesc) * descs.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_descs, descs.data(), sizeof(lbm3::BatchDesc) * descs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "lbm3_batch_create: %s\n", cudaGetErrorString(e));
    cudaGetLastError();
    destroy_batch(b);
    return LBM3_ECUDA;
  }
  *out = b;
  return LBM3_OK;
}

int32_t lbm3_batch_count(const lbm3_batch* b) { return b ? static_cast<int32_t>(b->ctx.size()) : -1; }

lbm3_status lbm3_batch_autotune(lbm3_batch* b, int32_t candidates, int32_t steps, int32_t* rows_out,
                                double* ms_out, double* table) {
  if (!b) return LBM3_EINVAL;
  if (candidates < 1 || candidates > 16 || steps < 1)
    return bfail(b, LBM3_EINVAL, "lbm3_batch_autotune: need 1 <= candidates <= 16 and steps >= 1");
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (!b->ctx[i]->state_set) return bfail(b, LBM3_ESTATE, "lbm3_batch_autotune: instance %zu not initialised", i);
    if (b->ctx[i]->in_shadow)
      return bfail(b, LBM3_ESTATE, "lbm3_batch_autotune: instance %zu holds populations set since the last step; "
                   "a reduced-state batch is tuned after a step", i);
  }
  DeviceGuard g(b->device);
  // candidates: the model's best-ranked heights, then 64 and 128 if absent
  std::vector<int> cand(b->ranked.begin(), b->ranked.begin() + std::min<size_t>(candidates, b->ranked.size()));
  for (int extra : {64, 128})
    if (std::find(cand.begin(), cand.end(), extra) == cand.end()) cand.push_back(extra);
  // every timed launch reads the current state and writes the idle buffers,
  // so neither the state nor the time changes
  const int parity = b->ctx[0]->cur;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return bfail(b, LBM3_ECUDA, "lbm3_batch_autotune: cannot create events");
  }
  int best_rows = b->rows;
  double best_ms = 1e300;
  lbm3_status st = LBM3_OK;
  for (size_t k = 0; k < cand.size() && st == LBM3_OK; ++k) {
    std::vector<lbm3::BatchItem> items;
    batch_items(b, cand[k], &items);
    st = batch_upload(b, items);
    if (st != LBM3_OK) break;
    st = launch_one(b, parity, b->stream);  // warm-up launch
    if (st != LBM3_OK) break;
    cudaEventRecord(e0, b->stream);
    for (int s = 0; s < steps && st == LBM3_OK; ++s) st = launch_one(b, parity, b->stream);
    cudaEventRecord(e1, b->stream);
    if (st != LBM3_OK) break;
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = bfail(b, LBM3_ECUDA, "lbm3_batch_autotune: %s", cudaGetErrorString(e));
      break;
    }
    const double per = static_cast<double>(ms) / steps;
    if (table) {
      table[2 * k] = cand[k];
      table[2 * k + 1] = per;
    }
    if (per < best_ms) {
      best_ms = per;
      best_rows = cand[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (table)
    for (size_t k = cand.size(); k < static_cast<size_t>(candidates) + 2; ++k) table[2 * k] = table[2 * k + 1] = 0.0;
  // keep the winner; the step graphs are captured again for its work list
  std::vector<lbm3::BatchItem> items;
  batch_items(b, best_rows, &items);
  const lbm3_status st2 = batch_upload(b, items);
  if (st == LBM3_OK) st = st2;
  b->rows = best_rows;
  for (int p = 0; p < 2; ++p)
    if (b->graph[p]) {
      cudaGraphExecDestroy(b->graph[p]);
      b->graph[p] = nullptr;
    }
  if (rows_out) *rows_out = best_rows;
  if (ms_out) *ms_out = best_ms;
  if (st != LBM3_OK) return st;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    st = check_device_errors(b->ctx[i]);
    if (st != LBM3_OK) return bcheck(b, st, static_cast<int>(i));
  }
  return LBM3_OK;
}

int32_t lbm3_batch_work_items(const lbm3_batch* b) { return b ? b->nitems : -1; }

lbm3_status lbm3_batch_init(lbm3_batch* b, int32_t i, const double* rho, int on_device) {
  if (!b) return LBM3_EINVAL;
  if (i < 0 || i >= static_cast<int32_t>(b->ctx.size())) return bfail(b, LBM3_EINVAL, "lbm3_batch_init: index %d", i);
  return bcheck(b, lbm3_init(b->ctx[i], rho, on_device), i);
}

lbm3_status lbm3_batch_set_populations(lbm3_batch* b, int32_t i, const double* f, int on_device) {
  if (!b) return LBM3_EINVAL;
  if (i < 0 || i >= static_cast<int32_t>(b->ctx.size()))
    return bfail(b, LBM3_EINVAL, "lbm3_batch_set_populations: index %d", i);
  return bcheck(b, lbm3_set_populations(b->ctx[i], f, on_device), i);
}

lbm3_status lbm3_batch_step(lbm3_batch* b, int64_t n) {
  if (!b) return LBM3_EINVAL;
  if (n < 0) return bfail(b, LBM3_EINVAL, "lbm3_batch_step: n < 0");
  for (size_t i = 0; i < b->ctx.size(); ++i)
    if (!b->ctx[i]->state_set) return bfail(b, LBM3_ESTATE, "lbm3_batch_step: instance %zu not initialised", i);
  DeviceGuard g(b->device);
  auto advance = [&](int64_t k) {
    for (lbm3_ctx* c : b->ctx) {
      if (k & 1) c->cur ^= 1;
      c->t += k;
    }
    b->t += k;
  };
  if (b->storage == LBM3_REDUCED && n > 0) {
    bool any = false;
    for (const lbm3_ctx* c : b->ctx) any = any || c->in_shadow;
    if (any) {
      lbm3_status st = batch_first_reduced_step(b, b->ctx[0]->cur);
      if (st != LBM3_OK) return st;
      advance(1);
      n -= 1;
    }
  }
  const int parity = b->ctx[0]->cur;
  if (n >= 2) {
    if (!b->graph[parity]) {
      lbm3_status st = build_graph(b, parity);
      if (st != LBM3_OK) return st;
    }
    for (int64_t k = 0; k < n / 2; ++k) {
      const cudaError_t e = cudaGraphLaunch(b->graph[parity], b->stream);
      if (e != cudaSuccess) return bfail(b, LBM3_ECUDA, "lbm3_batch_step: %s", cudaGetErrorString(e));
    }
    advance(n / 2 * 2);
  }
  if (n & 1) {
    lbm3_status st = launch_one(b, b->ctx[0]->cur, b->stream);
    if (st != LBM3_OK) return st;
    advance(1);
  }
  return LBM3_OK;
}

lbm3_status lbm3_batch_fields(lbm3_batch* b, int32_t i, double* rho, double* ux, double* uy, double* p,
                              int on_device) {
  if (!b) return LBM3_EINVAL;
  if (i < 0 || i >= static_cast<int32_t>(b->ctx.size()))
    return bfail(b, LBM3_EINVAL, "lbm3_batch_fields: index %d", i);
  return bcheck(b, lbm3_fields(b->ctx[i], rho, ux, uy, p, on_device), i);
}

lbm3_status lbm3_batch_populations(lbm3_batch* b, int32_t i, double* f, int on_device) {
  if (!b) return LBM3_EINVAL;
  if (i < 0 || i >= static_cast<int32_t>(b->ctx.size()))
    return bfail(b, LBM3_EINVAL, "lbm3_batch_populations: index %d", i);
  return bcheck(b, lbm3_populations(b->ctx[i], f, on_device), i);
}

lbm3_status lbm3_batch_mass(lbm3_batch* b, int32_t i, double* mass, double* mom) {
  if (!b) return LBM3_EINVAL;
  if (i < 0 || i >= static_cast<int32_t>(b->ctx.size())) return bfail(b, LBM3_EINVAL, "lbm3_batch_mass: index %d", i);
  return bcheck(b, lbm3_mass(b->ctx[i], mass, mom), i);
}

lbm3_status lbm3_batch_sync(lbm3_batch* b) {
  if (!b) return LBM3_EINVAL;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    lbm3_status st = lbm3_sync(b->ctx[i]);
    if (st != LBM3_OK) return bcheck(b, st, static_cast<int>(i));
  }
  return LBM3_OK;
}

int64_t lbm3_batch_time(const lbm3_batch* b) { return b ? b->t : -1; }

lbm3_status lbm3_batch_destroy(lbm3_batch* b) {
  if (!b) return LBM3_OK;
  DeviceGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  destroy_batch(b);
  return LBM3_OK;
}

const char* lbm3_batch_last_error(const lbm3_batch* b) { return b ? b->msg.c_str() : kNullBatchMsg; }

}  // extern "C"
