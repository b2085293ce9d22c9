// FP64 interface diagnostics of a state: the contact angles of Eq. theta_kl
// at the three-phase junctions of a droplet and the bulk pressures behind
// the Laplace jumps (Eq. laplace, Eq. 22).  The paper measures both but gives
// no procedure; the measurement defined here is:
//
//  * Interface points of a pair (k, l), m the third colour: on every link
//    (x, y)-(x+1, y) and (x, y)-(x, y+1) inside the grid (not across the
//    periodic edges) with phi_k, phi_l > 0 at both ends, where
//    s = ln(phi_k / phi_l) changes sign (s > 0 at exactly one end) and
//    phi_m < third_max at both ends: the zero of the linear interpolant of s.
//    Across the tanh profile of Eq. 21, ln(phi_k / phi_l) is linear in the
//    distance to the interface, so the point is exact there.
//  * Per pair, the circle minimising sum (x^2 + y^2 + D x + E y + F)^2 over
//    its points (algebraic fit), from nine FP64 moments of the points taken
//    relative to the grid centre.
//  * Junctions: the two intersections of the 1-2 and 1-3 circles; each
//    intersection of the 1-2/2-3 and 1-3/2-3 circles joins the nearer one;
//    a junction is the mean of its points.  At a junction each circle's
//    tangent is a line; one direction per line is taken such that no
//    half-plane holds all three (the configuration in which the three
//    tensions can balance, as in the Neumann triangle), the angle inside
//    fluid m is the angle between the directions of interfaces k-m and l-m,
//    and varphi_kl = 180 deg minus it.  The two junctions are averaged.
//  * Bulk pressure of fluid k: the mean of p = rho/3 over nodes with
//    phi_k > bulk_min.
//
// The O(N) part (points, moments, bulk sums) runs on the device in FP64 from
// the FP64 fields; the O(1) geometry runs on the host in FP64.  Partial sums
// are per block and added in block order, so results do not depend on
// scheduling.

#include <cmath>
#include <cstring>

#include "lbm3_internal.h"

namespace lbm3 {
namespace {

constexpr int kDiagThreads = 256;
constexpr int kDiagVals = 33;  // 3 pairs x 9 moments, then 3 fluids x (count, sum p)

__device__ __forceinline__ void add_point(double* acc, int q, double px, double py) {
  const double r2 = px * px + py * py;
  double* m = acc + 9 * q;
  m[0] += 1.0;
  m[1] += px;
  m[2] += py;
  m[3] += px * px;
  m[4] += px * py;
  m[5] += py * py;
  m[6] += px * r2;
  m[7] += py * r2;
  m[8] += r2;
}

// colour fractions of node n from the FP64 densities
__device__ __forceinline__ void fractions(const double* __restrict__ rho, size_t N, size_t n, double* ph) {
  const double a = rho[n], b = rho[N + n], c = rho[2 * N + n];
  const double r = (a + b) + c;
  ph[0] = a / r;
  ph[1] = b / r;
  ph[2] = c / r;
}

__global__ void __launch_bounds__(kDiagThreads) diag_partial_kernel(const double* __restrict__ rho,
                                                                    const double* __restrict__ p, int nx, int ny,
                                                                    double third_max, double bulk_min,
                                                                    double* __restrict__ partial) {
  double acc[kDiagVals];
#pragma unroll
  for (int j = 0; j < kDiagVals; ++j) acc[j] = 0.0;
  const size_t N = static_cast<size_t>(nx) * ny;
  const double ox = 0.5 * nx, oy = 0.5 * ny;
  const int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2};
  for (size_t n = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; n < N;
       n += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(n % nx), y = static_cast<int>(n / nx);
    double pa[3];
    fractions(rho, N, n, pa);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (pa[k] > bulk_min) {
        acc[27 + 2 * k] += 1.0;
        acc[28 + 2 * k] += p[n];
      }
#pragma unroll
    for (int axis = 0; axis < 2; ++axis) {  // link to (x+1, y), then to (x, y+1)
      if (axis == 0 ? x + 1 >= nx : y + 1 >= ny) continue;
      const size_t nb = axis == 0 ? n + 1 : n + nx;
      double pb[3];
      fractions(rho, N, nb, pb);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int k = pk[q], l = pl[q], m = 3 - k - l;
        if (!(pa[k] > 0.0 && pa[l] > 0.0 && pb[k] > 0.0 && pb[l] > 0.0)) continue;
        if (!(pa[m] < third_max && pb[m] < third_max)) continue;
        const double ra = pa[k] / pa[l], rb = pb[k] / pb[l];
        // ln r > 0 exactly when r > 1: the logarithms are only taken at crossings
        if ((ra > 1.0) == (rb > 1.0)) continue;
        const double sa = log(ra), sb = log(rb);
        const double t = sa / (sa - sb);
        const double px = (axis == 0 ? x + t : static_cast<double>(x)) - ox;
        const double py = (axis == 0 ? static_cast<double>(y) : y + t) - oy;
        add_point(acc, q, px, py);
      }
    }
  }
  // block sum: warp shuffles, then one row per warp in shared memory
  __shared__ double sh[kDiagThreads / 32][kDiagVals];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kDiagVals; ++j) {
    double v = acc[j];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sh[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagVals) {
    double v = 0.0;
    for (int w = 0; w < kDiagThreads / 32; ++w) v += sh[w][threadIdx.x];
    partial[static_cast<size_t>(blockIdx.x) * kDiagVals + threadIdx.x] = v;
  }
}

__global__ void diag_final_kernel(const double* __restrict__ partial, int blocks, double* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= kDiagVals) return;
  double v = 0.0;
  for (int b = 0; b < blocks; ++b) v += partial[static_cast<size_t>(b) * kDiagVals + j];
  out[j] = v;
}

// ------------------------------------------------------------ host geometry

struct Circle {
  double cx, cy, R;
  bool ok;
};

// Least-squares circle from the moments (n, Sx, Sy, Sxx, Sxy, Syy, Sxr2,
// Syr2, Sr2): the normal equations of min sum (r^2 + D x + E y + F)^2,
// solved by Gaussian elimination with partial pivoting.
Circle circle_from_moments(const double* m) {
  Circle c{0.0, 0.0, 0.0, false};
  if (m[0] < 3.0) return c;
  double A[3][4] = {{m[3], m[4], m[1], -m[6]}, {m[4], m[5], m[2], -m[7]}, {m[1], m[2], m[0], -m[8]}};
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (A[piv][col] == 0.0) return c;
    if (piv != col)
      for (int j = 0; j < 4; ++j) std::swap(A[piv][j], A[col][j]);
    for (int r = col + 1; r < 3; ++r) {
      const double f = A[r][col] / A[col][col];
      for (int j = col; j < 4; ++j) A[r][j] -= f * A[col][j];
    }
  }
  double s[3];
  for (int r = 2; r >= 0; --r) {
    double v = A[r][3];
    for (int j = r + 1; j < 3; ++j) v -= A[r][j] * s[j];
    s[r] = v / A[r][r];
  }
  c.cx = -0.5 * s[0];
  c.cy = -0.5 * s[1];
  const double R2 = c.cx * c.cx + c.cy * c.cy - s[2];
  if (!(R2 > 0.0)) return c;
  c.R = std::sqrt(R2);
  c.ok = true;
  return c;
}

// Intersections of two circles; returns how many (0 or 2).
int intersect(const Circle& a, const Circle& b, double P[2][2]) {
  const double dx = b.cx - a.cx, dy = b.cy - a.cy;
  const double d = std::hypot(dx, dy);
  if (d == 0.0 || d > a.R + b.R || d < std::fabs(a.R - b.R)) return 0;
  const double al = (a.R * a.R - b.R * b.R + d * d) / (2.0 * d);
  const double h = std::sqrt(std::fmax(a.R * a.R - al * al, 0.0));
  const double ux = dx / d, uy = dy / d;
  const double bx = a.cx + al * ux, by = a.cy + al * uy;
  P[0][0] = bx - h * uy;
  P[0][1] = by + h * ux;
  P[1][0] = bx + h * uy;
  P[1][1] = by - h * ux;
  return 2;
}

}  // namespace

size_t diag_scratch_doubles() { return static_cast<size_t>(kDiagMaxBlocks) * kDiagVals + kDiagVals; }

cudaError_t launch_diag(const double* rho, const double* p, int nx, int ny, double third_max, double bulk_min,
                        double* scratch, cudaStream_t s) {
  const size_t N = static_cast<size_t>(nx) * ny;
  size_t blocks = (N + kDiagThreads * 16 - 1) / (kDiagThreads * 16);
  if (blocks < 1) blocks = 1;
  if (blocks > static_cast<size_t>(kDiagMaxBlocks)) blocks = kDiagMaxBlocks;
  double* out = scratch + static_cast<size_t>(kDiagMaxBlocks) * kDiagVals;
  diag_partial_kernel<<<static_cast<int>(blocks), kDiagThreads, 0, s>>>(rho, p, nx, ny, third_max, bulk_min,
                                                                         scratch);
  diag_final_kernel<<<1, 64, 0, s>>>(scratch, static_cast<int>(blocks), out);
  return cudaGetLastError();
}

void diag_geometry(const double* sums, int nx, int ny, DiagResult* r) {
  std::memset(r, 0, sizeof *r);
  const double nan = std::nan("");
  const double ox = 0.5 * nx, oy = 0.5 * ny;
  Circle c[3];
  for (int q = 0; q < 3; ++q) {
    r->points[q] = sums[9 * q];
    c[q] = circle_from_moments(sums + 9 * q);
    if (!c[q].ok) r->flags |= 1;
    r->circle[q][0] = c[q].ok ? c[q].cx + ox : nan;
    r->circle[q][1] = c[q].ok ? c[q].cy + oy : nan;
    r->circle[q][2] = c[q].ok ? c[q].R : nan;
  }
  for (int k = 0; k < 3; ++k) {
    r->n_bulk[k] = sums[27 + 2 * k];
    r->p_bulk[k] = r->n_bulk[k] > 0.0 ? sums[28 + 2 * k] / r->n_bulk[k] : nan;
  }
  for (int j = 0; j < 2; ++j)
    for (int a = 0; a < 3; ++a) r->varphi_junction[j][a] = nan;
  for (int a = 0; a < 3; ++a) r->varphi[a] = nan;
  for (int j = 0; j < 2; ++j) r->junction[j][0] = r->junction[j][1] = nan;
  if (r->flags) return;
  double J[2][2];
  if (intersect(c[0], c[1], J) != 2) {
    r->flags |= 2;
    return;
  }
  double gsum[2][2] = {{J[0][0], J[0][1]}, {J[1][0], J[1][1]}};
  int gcount[2] = {1, 1};
  const int others[2][2] = {{0, 2}, {1, 2}};
  for (int o = 0; o < 2; ++o) {
    double P[2][2];
    if (intersect(c[others[o][0]], c[others[o][1]], P) != 2) continue;
    for (int i = 0; i < 2; ++i) {
      const double d0 = std::hypot(P[i][0] - J[0][0], P[i][1] - J[0][1]);
      const double d1 = std::hypot(P[i][0] - J[1][0], P[i][1] - J[1][1]);
      const int g = d1 < d0 ? 1 : 0;
      gsum[g][0] += P[i][0];
      gsum[g][1] += P[i][1];
      gcount[g] += 1;
    }
  }
  const double pi = std::acos(-1.0);
  double mean[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < 2; ++j) {
    const double jx = gsum[j][0] / gcount[j], jy = gsum[j][1] / gcount[j];
    r->junction[j][0] = jx + ox;
    r->junction[j][1] = jy + oy;
    double line[3][2];
    for (int q = 0; q < 3; ++q) {  // tangent of circle q at the junction
      const double vx = -(jy - c[q].cy), vy = jx - c[q].cx;
      const double nv = std::hypot(vx, vy);
      line[q][0] = vx / nv;
      line[q][1] = vy / nv;
    }
    // directions: the first line as it is; signs of the other two such
    // that every gap between consecutive directions is below pi
    bool found = false;
    double ray[3][2];
    for (int s2 = 0; s2 < 2 && !found; ++s2)
      for (int s3 = 0; s3 < 2 && !found; ++s3) {
        const double sg[3] = {1.0, s2 ? -1.0 : 1.0, s3 ? -1.0 : 1.0};
        double ang[3];
        for (int q = 0; q < 3; ++q) {
          ray[q][0] = sg[q] * line[q][0];
          ray[q][1] = sg[q] * line[q][1];
          ang[q] = std::atan2(ray[q][1], ray[q][0]);
        }
        double lo = std::fmin(ang[0], std::fmin(ang[1], ang[2]));
        double hi = std::fmax(ang[0], std::fmax(ang[1], ang[2]));
        double mid = ang[0] + ang[1] + ang[2] - lo - hi;
        const double gmax = std::fmax(std::fmax(mid - lo, hi - mid), 2.0 * pi - (hi - lo));
        found = gmax < pi;
      }
    if (!found) {
      r->flags |= 4;
      return;
    }
    auto angle = [&](int a, int b) {
      double d = ray[a][0] * ray[b][0] + ray[a][1] * ray[b][1];
      d = d > 1.0 ? 1.0 : (d < -1.0 ? -1.0 : d);
      return std::acos(d) * 180.0 / pi;
    };
    // inside fluid 3 between 1-3 and 2-3; inside 2 between 1-2 and 2-3; inside 1 between 1-2 and 1-3
    r->varphi_junction[j][0] = 180.0 - angle(1, 2);
    r->varphi_junction[j][1] = 180.0 - angle(0, 2);
    r->varphi_junction[j][2] = 180.0 - angle(0, 1);
    for (int a = 0; a < 3; ++a) mean[a] += 0.5 * r->varphi_junction[j][a];
  }
  for (int a = 0; a < 3; ++a) r->varphi[a] = mean[a];
}

}  // namespace lbm3
