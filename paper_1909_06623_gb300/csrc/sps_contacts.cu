// Contact set (Sec. 3.2), the contact Jacobian D and its transpose
// (eq. Dmatdef, eq. Dtranspose), the BBPGD statistics of Algorithm 1, and the
// BBPGD iteration for the identity mobility.
//
// Contact search.  Small suspensions test every pair i < j.  Large ones use a
// uniform grid of cells whose side is at least 2 max a_c + delta, so that every
// contact pair lies in the same or in adjacent cells; spheres are sorted by
// cell (stable radix sort), and each sphere scans the 3 x 3 rows of adjacent
// cells, which are contiguous runs of the sorted order.  Candidates are
// screened in FP32 with a margin that bounds the rounding of the FP32 copies;
// every survivor takes the FP64 test of the all-pairs search (sps_contact_test)
// and each row is sorted by j, so both searches give the same list to the bit.
//
// D and D^T: per sphere, its incident contacts in contact order (a stable sort
// of the contact ends); per contact, n . (U_j - U_i).  All reductions use a
// fixed partition and order, so every result is reproducible run to run.

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sps_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kStatBlocks = 8 * 152;   // fixed partition of the BBPGD reductions
constexpr int kBoundBlocks = 2 * 152;

inline int nblk(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ bool contact_at(const double* pos, const double* rad, double acs,
                                           double delta, double drel, int i, int j, SpsContactGeom* g) {
  return sps_contact_test(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], rad[i], pos[3 * j],
                          pos[3 * j + 1], pos[3 * j + 2], rad[j], acs, delta, drel, g);
}

// ---------------------------------------------------------------------------
// all pairs
// ---------------------------------------------------------------------------
__global__ void k_pairs_count(int N, const double* pos, const double* rad, double acs, double delta,
                              double drel, int* cnt, int* cnt2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c = 0;
  for (int j = i + 1; j < N; ++j)
    if (contact_at(pos, rad, acs, delta, drel, i, j, nullptr)) {
      ++c;
      atomicAdd(&cnt2[j], 1);   // integer count of contacts where j is second
    }
  cnt[i] = c;
}

__global__ void k_pairs_fill(int N, const double* pos, const double* rad, double acs, double delta,
                             double drel, const int* ptr, int* ij) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int o = ptr[i];
  for (int j = i + 1; j < N; ++j)
    if (contact_at(pos, rad, acs, delta, drel, i, j, nullptr)) {
      ij[2 * o] = i;
      ij[2 * o + 1] = j;
      ++o;
    }
}

// Phi and the normal of every listed contact (one thread per contact, the
// arithmetic of the contact test), and the contact ends for the incidence sort
__global__ void k_contact_geom(int nc, const int* __restrict__ ij, const double* __restrict__ pos,
                               const double* __restrict__ rad, double acs, double* __restrict__ phi,
                               double* __restrict__ nrm) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nc) return;
  const int i = ij[2 * l], j = ij[2 * l + 1];
  SpsContactGeom g;
  // delta = +inf: the same rounded operations, and the geometry is always written
  contact_at(pos, rad, acs, INFINITY, 0.0, i, j, &g);
  phi[l] = g.phi;
  nrm[3 * l + 0] = g.nx;
  nrm[3 * l + 1] = g.ny;
  nrm[3 * l + 2] = g.nz;
}

// ---------------------------------------------------------------------------
// cell list
// ---------------------------------------------------------------------------
// per block: min x, y, z, max x, y, z, max a, number of bad inputs
__global__ void k_cl_bounds(int N, const double* __restrict__ pos, const double* __restrict__ rad,
                            double* __restrict__ part) {
  double v[8] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], a = rad[i];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(a) || !(a > 0)) {
      v[7] += 1.0;
      continue;
    }
    v[0] = fmin(v[0], x);
    v[1] = fmin(v[1], y);
    v[2] = fmin(v[2], z);
    v[3] = fmax(v[3], x);
    v[4] = fmax(v[4], y);
    v[5] = fmax(v[5], z);
    v[6] = fmax(v[6], a);
  }
  __shared__ double red[kThreads / 32][8];
#pragma unroll
  for (int c = 0; c < 8; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v[c], o);
      v[c] = c < 3 ? fmin(v[c], w) : (c < 7 ? fmax(v[c], w) : v[c] + w);
    }
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 8; ++c) red[threadIdx.x >> 5][c] = v[c];
  __syncthreads();
  if (threadIdx.x < 8) {
    const int c = threadIdx.x;
    double s = red[0][c];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      s = c < 3 ? fmin(s, red[w][c]) : (c < 7 ? fmax(s, red[w][c]) : s + red[w][c]);
    part[c * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_cl_bounds_finish(int nb, const double* __restrict__ part, double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= 8) return;
  double s = part[c * nb];
  for (int b = 1; b < nb; ++b) {
    const double w = part[c * nb + b];
    s = c < 3 ? fmin(s, w) : (c < 7 ? fmax(s, w) : s + w);
  }
  out[c] = s;
}

struct CellGrid {
  double lo[3], inv_w[3];
  int dims[3];
  float eps;   // absolute margin of the FP32 screen
};

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_w, int dim) {
  const int c = (int)((x - lo) * inv_w);
  return min(max(c, 0), dim - 1);
}

__global__ void k_cl_keys(int N, const double* __restrict__ pos, CellGrid G, int* __restrict__ key,
                          int* __restrict__ id) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int cx = cell_coord(pos[3 * s], G.lo[0], G.inv_w[0], G.dims[0]);
  const int cy = cell_coord(pos[3 * s + 1], G.lo[1], G.inv_w[1], G.dims[1]);
  const int cz = cell_coord(pos[3 * s + 2], G.lo[2], G.inv_w[2], G.dims[2]);
  key[s] = (cz * G.dims[1] + cy) * G.dims[0] + cx;
  id[s] = s;
}

// start[c] = first sorted position whose cell is >= c, for c = 0..ncells

// sorted copies: FP32 (x, y, z relative to the grid origin, a), FP64 (x, y, z, a)
__global__ void k_cl_gather(int N, const int* __restrict__ id, const double* __restrict__ pos,
                            const double* __restrict__ rad, CellGrid G, float4* __restrict__ cf,
                            double4_32a* __restrict__ cd) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int s = id[k];
  const double x = pos[3 * s], y = pos[3 * s + 1], z = pos[3 * s + 2], a = rad[s];
  cf[k] = make_float4((float)(x - G.lo[0]), (float)(y - G.lo[1]), (float)(z - G.lo[2]), (float)a);
  cd[k] = make_double4_32a(x, y, z, a);
}

// Visits every sphere j > i in the 27 cells around sorted position k that can
// satisfy the contact test; f(i, j) is called for each pair that passes it.
// The FP32 screen decides a pair when its FP32 distance is clearly above
// (a_c,i + a_c,j + delta_l)(1 + 1e-5) + eps or clearly below
// (a_c,i + a_c,j + delta_l)(1 - 1e-5) - eps, eps bounding the rounding of the
// FP32 coordinates; only pairs in that band take the FP64 test, so every
// decision equals the FP64 test's.
template <class F>
__device__ __forceinline__ void cl_scan(int k, const int* __restrict__ key, const int* __restrict__ id,
                                        const float4* __restrict__ cf, const double4_32a* __restrict__ cd,
                                        const int* __restrict__ start, const CellGrid& G, float acsf,
                                        float deltaf, float drelf, double acs, double delta,
                                        double drel, F f) {
  const int i = id[k];
  const float4 me = cf[k];
  const double4_32a md = cd[k];
  const int kk = key[k];
  const int cx = kk % G.dims[0], cy = (kk / G.dims[0]) % G.dims[1], cz = kk / (G.dims[0] * G.dims[1]);
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, G.dims[0] - 1);
  for (int zz = max(cz - 1, 0); zz <= min(cz + 1, G.dims[2] - 1); ++zz)
    for (int yy = max(cy - 1, 0); yy <= min(cy + 1, G.dims[1] - 1); ++yy) {
      const int row = (zz * G.dims[1] + yy) * G.dims[0];
      const int m1 = start[row + x1 + 1];
      for (int m = start[row + x0]; m < m1; ++m) {
        const int j = id[m];
        if (j <= i) continue;
        const float4 o = cf[m];
        const float dx = o.x - me.x, dy = o.y - me.y, dz = o.z - me.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float tn = fmaf(acsf + drelf, me.w + o.w, deltaf);
        const float hi = fmaf(tn, 1.00001f, G.eps);
        if (d2 > hi * hi) continue;                   // certainly apart
        const float lo = fmaf(tn, 0.99999f, -G.eps);
        if (lo > 0.f && d2 < lo * lo) {               // certainly in contact
          f(i, j);
          continue;
        }
        const double4_32a od = cd[m];                 // near the threshold: FP64 test
        if (sps_contact_test(md.x, md.y, md.z, md.w, od.x, od.y, od.z, od.w, acs, delta, drel, nullptr))
          f(i, j);
      }
    }
}

__global__ void __launch_bounds__(kThreads) k_cl_count(int N, const int* __restrict__ key,
                                                      const int* __restrict__ id,
                                                      const float4* __restrict__ cf,
                                                      const double4_32a* __restrict__ cd,
                                                      const int* __restrict__ start, CellGrid G,
                                                      double acs, double delta, double drel,
                                                      int* __restrict__ cnt, int* __restrict__ cnt2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int c = 0;
  cl_scan(k, key, id, cf, cd, start, G, (float)acs, (float)delta, (float)drel, acs, delta, drel,
          [&](int, int j) {
    ++c;
    atomicAdd(&cnt2[j], 1);
  });
  cnt[id[k]] = c;
}

// writes row i: (i, j) for the j's found, sorted ascending in place
__global__ void __launch_bounds__(kThreads) k_cl_fill(int N, const int* __restrict__ key,
                                                     const int* __restrict__ id,
                                                     const float4* __restrict__ cf,
                                                     const double4_32a* __restrict__ cd,
                                                     const int* __restrict__ start, CellGrid G,
                                                     double acs, double delta, double drel,
                                                     const int* __restrict__ ptr, int* __restrict__ ij) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int i = id[k];
  const int o0 = ptr[i], oe = ptr[i + 1];
  int o = o0;
  // the count pass applied the same predicate, so the row fills [o0, oe)
  // exactly; the bound only keeps every store inside the row regardless
  cl_scan(k, key, id, cf, cd, start, G, (float)acs, (float)delta, (float)drel, acs, delta, drel,
          [&](int, int j) {
    if (o < oe) ij[2 * o + 1] = j;
    ++o;
  });
  o = min(o, oe);
  for (int t = o0 + 1; t < o; ++t) {   // insertion sort of the row by j
    const int v = ij[2 * t + 1];
    int u = t;
    while (u > o0 && ij[2 * (u - 1) + 1] > v) {
      ij[2 * u + 1] = ij[2 * (u - 1) + 1];
      --u;
    }
    ij[2 * u + 1] = v;
  }
  for (int t = o0; t < o; ++t) ij[2 * t] = i;
}

__global__ void k_add_counts(int N, const int* a, const int* b, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = a[i] + b[i];
}

// wall contacts per sphere (entry n set to 0 for the scan), and their rows:
// (-1 - w, i), Phi, the wall normal, sorted by (sphere, wall)
__global__ void k_wall_count(int n, const double* __restrict__ pos, const double* __restrict__ rad, SpsWalls W,
                             double acs, double delta, double drel, int* __restrict__ wcnt,
                             int* __restrict__ inc_cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    wcnt[n] = 0;
    return;
  }
  int c = 0;
  double ph;
  for (int w = 0; w < W.n; ++w)
    if (sps_wall_test(W.w[w], pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], rad[i], acs, delta, drel, &ph)) ++c;
  wcnt[i] = c;
  inc_cnt[i] += c;
}

__global__ void k_wall_fill(int n, const double* __restrict__ pos, const double* __restrict__ rad, SpsWalls W,
                            double acs, double delta, double drel, const int* __restrict__ wptr, int base,
                            int* __restrict__ ij, double* __restrict__ phi, double* __restrict__ nrm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = base + wptr[i];
  double ph;
  for (int w = 0; w < W.n; ++w)
    if (sps_wall_test(W.w[w], pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], rad[i], acs, delta, drel, &ph)) {
      ij[2 * o] = -1 - w;
      ij[2 * o + 1] = i;
      phi[o] = ph;
      nrm[3 * o + 0] = W.w[w][0];
      nrm[3 * o + 1] = W.w[w][1];
      nrm[3 * o + 2] = W.w[w][2];
      ++o;
    }
}

// ---------------------------------------------------------------------------
// D and D^T
// ---------------------------------------------------------------------------
// F_c = D gamma: per sphere, its incident contacts in contact order
__global__ void k_D(int N, const int* __restrict__ inc_ptr, const int* __restrict__ inc,
                    const double* __restrict__ nrm, const double* __restrict__ gam,
                    double* __restrict__ FT) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  double f0 = 0.0, f1 = 0.0, f2 = 0.0;
  for (int e = inc_ptr[s]; e < inc_ptr[s + 1]; ++e) {
    const int v = inc[e], l = v >> 1;
    const double g = gam[l];
    const double a0 = __dmul_rn(g, nrm[3 * l]), a1 = __dmul_rn(g, nrm[3 * l + 1]),
                 a2 = __dmul_rn(g, nrm[3 * l + 2]);
    if (v & 1) {
      f0 = __dadd_rn(f0, a0);
      f1 = __dadd_rn(f1, a1);
      f2 = __dadd_rn(f2, a2);
    } else {
      f0 = __dsub_rn(f0, a0);
      f1 = __dsub_rn(f1, a1);
      f2 = __dsub_rn(f2, a2);
    }
  }
  FT[6 * s + 0] = f0;
  FT[6 * s + 1] = f1;
  FT[6 * s + 2] = f2;
  FT[6 * s + 3] = 0.0;
  FT[6 * s + 4] = 0.0;
  FT[6 * s + 5] = 0.0;
}

// (D^T U)_l = n_l . (U_j - U_i)
__global__ void k_DT(int nc, const int* __restrict__ ij, const double* __restrict__ nrm,
                     const double* __restrict__ UO, double* __restrict__ out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nc) return;
  const int i = ij[2 * l], j = ij[2 * l + 1];
  double acc = 0.0;
  // a wall (first index negative) does not move
  for (int c = 0; c < 3; ++c) acc += nrm[3 * l + c] * (UO[6 * j + c] - (i >= 0 ? UO[6 * i + c] : 0.0));
  out[l] = acc;
}

// ---------------------------------------------------------------------------
// BBPGD statistics: [sum min(gam_n, g_n)^2, s.s, s.y, y.y, g_n.g_n] with
// s = gam_n - gam_o, y = g_n - g_o (Algorithm 1, eq. mmapnorm)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void stat_add(double a[5], double gn, double ggn, double go, double ggo,
                                         bool old) {
  const double mn = fmin(gn, ggn);
  a[0] += mn * mn;
  if (old) {
    const double s = gn - go, y = ggn - ggo;
    a[1] += s * s;
    a[2] += s * y;
    a[3] += y * y;
  }
  a[4] += ggn * ggn;
}

// block partial of the five sums into part[c * gridDim.x + blockIdx.x]
__device__ __forceinline__ void stat_store(double a[5], double* part) {
  __shared__ double red[kThreads / 32][5];
#pragma unroll
  for (int c = 0; c < 5; ++c)
    for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 5; ++c) red[threadIdx.x >> 5][c] = a[c];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    part[threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kThreads) k_bb_stats_part(int n, const double* __restrict__ gam_new,
                                                           const double* __restrict__ g_new,
                                                           const double* __restrict__ gam_old,
                                                           const double* __restrict__ g_old,
                                                           double* __restrict__ part) {
  double a[5] = {0, 0, 0, 0, 0};
  const bool old = gam_old != nullptr;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x)
    stat_add(a, gam_new[l], g_new[l], old ? gam_old[l] : 0.0, old ? g_old[l] : 0.0, old);
  stat_store(a, part);
}

// one warp per statistic: lane-strided partial sums, then a fixed shuffle tree
__global__ void k_stat_finish(int nb, const double* __restrict__ part, double* __restrict__ out) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= 5) return;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += part[c * nb + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = s;
}

// Identity mobility, one BBPGD iteration in three passes.  On this part FP64
// arithmetic, not memory, is the scarce resource, so each pass keeps whole
// warps busy, every FP64 operation is needed by the result, and comparisons
// run on the integer units:
//   1. per contact: gam_n = max(gam - alpha g, 0)                   (1 FMA)
//   2. per sphere:  F_s = sum of (+-gam_n) n over incident contacts (3 FMA each)
//   3. per contact: g_n = q + n . (F_j - F_i) and the statistics    (6 + 5)

// max(x, 0) on the bit pattern: a set sign bit gives +0 (a NaN stays a NaN)
__device__ __forceinline__ double clamp_pos(double x) {
  const long long b = __double_as_longlong(x);
  return __longlong_as_double(b & ~(b >> 63));
}

// min(x, y) by integer comparison of order-preserving keys (finite inputs)
__device__ __forceinline__ double min_bits(double x, double y) {
  const long long a = __double_as_longlong(x), b = __double_as_longlong(y);
  const long long ka = a ^ ((a >> 63) & 0x7FFFFFFFFFFFFFFFll);
  const long long kb = b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
  return (kb < ka) ? y : x;
}

__global__ void k_bb_proj(int nc, double alpha, const double* __restrict__ gam,
                          const double* __restrict__ g, double* __restrict__ gam_new) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < nc) gam_new[l] = clamp_pos(fma(-alpha, g[l], gam[l]));
}

// Per block of kThreads consecutive spheres, their order by decreasing number
// of incident contacts (ties by index): the gather below gives each warp
// spheres of about equal work, while a block still covers the same spheres.
__global__ void __launch_bounds__(kThreads) k_degree_order(int N, const int* __restrict__ inc_ptr,
                                                          int* __restrict__ order) {
  __shared__ int cnt[kThreads];
  const int s0 = blockIdx.x * kThreads, t = threadIdx.x, s = s0 + t;
  cnt[t] = (s < N) ? inc_ptr[s + 1] - inc_ptr[s] : -1;
  __syncthreads();
  if (s >= N) return;
  const int me = cnt[t];
  int rank = 0;
  for (int u = 0; u < kThreads; ++u) {
    const int c = cnt[u];
    rank += (c > me) || (c == me && u < t);
  }
  order[s0 + rank] = s;
}

__global__ void __launch_bounds__(kThreads) k_bb_gather(int N, const int* __restrict__ order,
                                                       const int* __restrict__ inc_ptr,
                                                       const int* __restrict__ inc,
                                                       const double* __restrict__ nrm,
                                                       const double* __restrict__ gam_new,
                                                       double* __restrict__ F3) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int s = order[k];
  double f0 = 0.0, f1 = 0.0, f2 = 0.0;
  const int e1 = inc_ptr[s + 1];
  for (int e = inc_ptr[s]; e < e1; ++e) {
    const int v = inc[e], l = v >> 1;
    // -gamma for the contact's first sphere: a sign-bit flip on the integer units
    const double gs = __longlong_as_double(__double_as_longlong(gam_new[l]) ^
                                           ((long long)(~v & 1) << 63));
    f0 = fma(gs, nrm[3 * l], f0);
    f1 = fma(gs, nrm[3 * l + 1], f1);
    f2 = fma(gs, nrm[3 * l + 2], f2);
  }
  F3[3 * s + 0] = f0;
  F3[3 * s + 1] = f1;
  F3[3 * s + 2] = f2;
}

// statistics [sum min(gam_n, g_n)^2, s.s, s.y, y.y (BB2 only), 0]
__global__ void __launch_bounds__(kThreads) k_bb_ident_DT(int nc, const int* __restrict__ ij,
                                                         const double* __restrict__ nrm,
                                                         const double* __restrict__ F3,
                                                         const double* __restrict__ q,
                                                         const double* __restrict__ gam_new,
                                                         const double* __restrict__ gam,
                                                         const double* __restrict__ g, int want_yy,
                                                         double* __restrict__ g_new,
                                                         double* __restrict__ part) {
  double a[5] = {0, 0, 0, 0, 0};
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nc; l += gridDim.x * blockDim.x) {
    const int i = ij[2 * l], j = ij[2 * l + 1];
    double acc = q[l];
    double fi0 = 0.0, fi1 = 0.0, fi2 = 0.0;   // a wall (first index negative) does not move
    if (i >= 0) {
      fi0 = F3[3 * i];
      fi1 = F3[3 * i + 1];
      fi2 = F3[3 * i + 2];
    }
    acc = fma(nrm[3 * l], F3[3 * j] - fi0, acc);
    acc = fma(nrm[3 * l + 1], F3[3 * j + 1] - fi1, acc);
    acc = fma(nrm[3 * l + 2], F3[3 * j + 2] - fi2, acc);
    g_new[l] = acc;
    const double gn = gam_new[l];
    const double mn = min_bits(gn, acc), sv = gn - gam[l], yv = acc - g[l];
    a[0] = fma(mn, mn, a[0]);
    a[1] = fma(sv, sv, a[1]);
    a[2] = fma(sv, yv, a[2]);
    if (want_yy) a[3] = fma(yv, yv, a[3]);
  }
  stat_store(a, part);
}

// dL/dc through the contact geometry of a collision step (Phi and the normals
// in D), per sphere over its incident active contacts l (first sphere -, second +):
//   v_l = (I - n n^T) t_l / |c_j - c_i| - (mu_l / dt) n_l,
//   t_l = gamma_l (w_j - w_i) - mu_l (U_j - U_i),  w = dL/dF, force parts
__global__ void k_contact_grad(int N, const int* __restrict__ inc_ptr, const int* __restrict__ inc,
                               const int* __restrict__ ij, const double* __restrict__ nrm,
                               const double* __restrict__ pos, const double* __restrict__ gam,
                               const double* __restrict__ mu, const double* __restrict__ w,
                               const double* __restrict__ U, double idt, double* __restrict__ dx) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int e = inc_ptr[s]; e < inc_ptr[s + 1]; ++e) {
    const int v = inc[e], l = v >> 1;
    if (!(gam[l] > 0.0)) continue;
    const int i = ij[2 * l], j = ij[2 * l + 1];
    const double nx = nrm[3 * l], ny = nrm[3 * l + 1], nz = nrm[3 * l + 2];
    const double dx0 = pos[3 * j] - pos[3 * i], dy0 = pos[3 * j + 1] - pos[3 * i + 1],
                 dz0 = pos[3 * j + 2] - pos[3 * i + 2];
    const double d = sqrt(dx0 * dx0 + dy0 * dy0 + dz0 * dz0);
    const double tx = gam[l] * (w[6 * j] - w[6 * i]) - mu[l] * (U[6 * j] - U[6 * i]);
    const double ty = gam[l] * (w[6 * j + 1] - w[6 * i + 1]) - mu[l] * (U[6 * j + 1] - U[6 * i + 1]);
    const double tz = gam[l] * (w[6 * j + 2] - w[6 * i + 2]) - mu[l] * (U[6 * j + 2] - U[6 * i + 2]);
    const double nt = nx * tx + ny * ty + nz * tz;
    const double c = mu[l] * idt;
    const double vx = (tx - nx * nt) / d - c * nx, vy = (ty - ny * nt) / d - c * ny,
                 vz = (tz - nz * nt) / d - c * nz;
    if (v & 1) {
      g0 += vx;
      g1 += vy;
      g2 += vz;
    } else {
      g0 -= vx;
      g1 -= vy;
      g2 -= vz;
    }
  }
  dx[3 * s] += g0;
  dx[3 * s + 1] += g1;
  dx[3 * s + 2] += g2;
}

__global__ void k_identity_U(int N, const double* __restrict__ FT, const double* __restrict__ F3,
                             double* __restrict__ UO) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6 * N) return;
  const int s = t / 6, c = t - 6 * s;
  UO[t] = FT[t] + ((F3 && c < 3) ? F3[3 * s + c] : 0.0);
}

// flags: 1 non-finite position or radius, 2 non-positive radius, 4 non-finite FT
__global__ void k_check(int N, const double* __restrict__ pos, const double* __restrict__ rad,
                        const double* __restrict__ FT, int* __restrict__ flag) {
  int f = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
    if (!isfinite(pos[3 * s]) || !isfinite(pos[3 * s + 1]) || !isfinite(pos[3 * s + 2]) ||
        !isfinite(rad[s]))
      f |= 1;
    if (!(rad[s] > 0)) f |= 2;
    if (FT)
      for (int c = 0; c < 6; ++c)
        if (!isfinite(FT[6 * s + c])) f |= 4;
  }
  if (f) atomicOr(flag, f);
}

__global__ void k_count_pos(int n, const double* __restrict__ v, int* __restrict__ out) {
  int c = 0;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) c += v[l] > 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ---------------------------------------------------------------------------
// exclusive scan of n ints (out may alias in): block scans of 4,096 elements,
// an exclusive scan of the block totals in one block, then the offsets added
// ---------------------------------------------------------------------------
constexpr int kScanT = 1024, kScanPer = 4, kScanTile = kScanT * kScanPer;

__device__ __forceinline__ int block_exclusive(int x, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int v = x;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const int ex = v - x + (warp ? wsum[warp - 1] : 0);
  *total = wsum[31];
  __syncthreads();
  return ex;
}

__global__ void __launch_bounds__(kScanT) k_scan_blocks(long long n, const int* in, int* out, int* tot) {
  __shared__ int wsum[32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
  int v[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int total;
  int run = block_exclusive(s, wsum, &total);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanT) k_scan_totals(int nb, int* tot) {
  __shared__ int wsum[32];
  const int per = (nb + kScanT - 1) / kScanT;
  const int a = min(nb, (int)threadIdx.x * per), b = min(nb, a + per);
  int s = 0;
  for (int i = a; i < b; ++i) s += tot[i];
  int total;
  int run = block_exclusive(s, wsum, &total);
  for (int i = a; i < b; ++i) {
    const int v = tot[i];
    tot[i] = run;
    run += v;
  }
}

__global__ void k_scan_add(long long n, int* out, const int* __restrict__ tot) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] += tot[i / kScanTile];
}

// ---------------------------------------------------------------------------
// cell list by counting sort (the order inside a cell is free: every row of
// the contact list is sorted by j afterwards)
// ---------------------------------------------------------------------------
__global__ void k_cell_hist(int N, const int* __restrict__ key, int* __restrict__ cnt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) atomicAdd(&cnt[key[k]], 1);
}
__global__ void k_cell_scatter(int N, const int* __restrict__ key, const int* __restrict__ id,
                               const int* __restrict__ start, int* __restrict__ fill, int* __restrict__ key2,
                               int* __restrict__ id2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int c = key[k];
  const int o = start[c] + atomicAdd(&fill[c], 1);
  key2[o] = c;
  id2[o] = id[k];
}

// ---------------------------------------------------------------------------
// incidence lists (each sphere's contact ends in contact order): sphere s
// is the second body of pair contacts in rows i < s (they come first in
// contact order), then the first body of its own row, then the second body
// of its wall contacts.  Rows and wall blocks are placed directly; the
// second-body ends arrive in any order and each sphere sorts them.
// ---------------------------------------------------------------------------
__global__ void k_inc_fill(int nc, int npair, const int* __restrict__ ij, const int* __restrict__ cptr,
                           const int* __restrict__ ccount, const int* __restrict__ ccount2,
                           const int* __restrict__ wptr, const int* __restrict__ inc_ptr,
                           int* __restrict__ fill2, int* __restrict__ inc) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nc) return;
  const int i = ij[2 * l], j = ij[2 * l + 1];
  if (l < npair) {
    inc[inc_ptr[i] + ccount2[i] + (l - cptr[i])] = 2 * l;
    inc[inc_ptr[j] + atomicAdd(&fill2[j], 1)] = 2 * l + 1;
  } else {
    inc[inc_ptr[j] + ccount2[j] + ccount[j] + (l - npair - wptr[j])] = 2 * l + 1;
  }
}
__global__ void k_inc_sort(int N, const int* __restrict__ inc_ptr, const int* __restrict__ ccount2,
                           int* __restrict__ inc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  int* a = inc + inc_ptr[s];
  const int m = ccount2[s];
  for (int t = 1; t < m; ++t) {
    const int v = a[t];
    int u = t;
    while (u > 0 && a[u - 1] > v) {
      a[u] = a[u - 1];
      --u;
    }
    a[u] = v;
  }
}

int read_int(sps_ctx* ctx, const int* d, int* h) {
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::memcpy(h, ctx->h_pinned, sizeof(int));
  return SPS_OK;
}

int exclusive_scan_impl(sps_ctx* ctx, const int* in, int* out, long long n) {
  if (n <= 0) return SPS_OK;
  const long long nb = (n + kScanTile - 1) / kScanTile;
  SPS_TRY(sps_grow(ctx, &ctx->d_scan_tot, ctx->cap_scan_tot, (size_t)nb + 1));
  k_scan_blocks<<<(int)nb, kScanT, 0, ctx->stream>>>(n, in, out, ctx->d_scan_tot);
  SPS_LAUNCHED(ctx);
  if (nb > 1) {
    k_scan_totals<<<1, kScanT, 0, ctx->stream>>>((int)nb, ctx->d_scan_tot);
    SPS_LAUNCHED(ctx);
    k_scan_add<<<(int)std::min<long long>((n + 255) / 256, 8 * 152), 256, 0, ctx->stream>>>(n, out,
                                                                                          ctx->d_scan_tot);
    SPS_LAUNCHED(ctx);
  }
  return SPS_OK;
}


// cell-list counts: cnt (as first sphere), cnt2 (as second) for n spheres
int cell_counts(sps_ctx* ctx, int n, const double* pos, const double* radii, CellGrid* Gout,
                int* ncells_out) {
  const double acs = ctx->prm.a_c_scale, delta = ctx->prm.delta, drel = ctx->prm.delta_rel;
  size_t cp = 0;
  if (!ctx->d_cl_part) SPS_TRY(sps_grow(ctx, &ctx->d_cl_part, cp, (size_t)8 * kBoundBlocks + 8));
  k_cl_bounds<<<kBoundBlocks, kThreads, 0, ctx->stream>>>(n, pos, radii, ctx->d_cl_part);
  SPS_LAUNCHED(ctx);
  double* bounds = ctx->d_cl_part + 8 * kBoundBlocks;
  k_cl_bounds_finish<<<1, 32, 0, ctx->stream>>>(kBoundBlocks, ctx->d_cl_part, bounds);
  SPS_LAUNCHED(ctx);
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, bounds, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double b[8];
  std::memcpy(b, ctx->h_pinned, sizeof(b));
  if (b[7] > 0) return sps_fail(ctx, SPS_ERR_NONFINITE, "contacts: positions or radii not finite and positive");
  // cell side >= 2 max a_c + max delta_l (with a relative margin over rounding)
  double h = (2.0 * (acs + drel) * b[6] + delta) * (1.0 + 1e-9);
  const long long cap_cells = std::min<long long>(1LL << 30, std::max<long long>(64, 2LL * n));
  CellGrid G;
  double ext[3], emax = 0.0;
  for (int d = 0; d < 3; ++d) {
    ext[d] = b[3 + d] - b[d];
    emax = std::max(emax, ext[d]);
  }
  long long dims[3];
  for (;;) {
    long long tot = 1;
    for (int d = 0; d < 3; ++d) {
      const double f = std::floor(ext[d] / h);
      dims[d] = (f >= 1.0) ? (long long)std::min(f, 1e9) : 1;
      tot *= dims[d];
      if (tot > cap_cells) break;
    }
    if (tot <= cap_cells) break;
    h *= 1.25;
  }
  for (int d = 0; d < 3; ++d) {
    G.lo[d] = b[d];
    G.dims[d] = (int)dims[d];
    // cell width ext / dims >= h: pairs closer than h land in adjacent cells
    G.inv_w[d] = dims[d] > 1 ? (double)dims[d] / ext[d] : 0.0;
  }
  // FP32 copies of coordinates relative to lo are within 2^-24 emax of the
  // FP64 values: the screen's absolute margin covers both ends with room
  G.eps = (float)(8.0 * emax * 5.9604644775390625e-8) + 1e-30f;
  const int ncells = G.dims[0] * G.dims[1] * G.dims[2];
  // buffers
  if ((size_t)n > ctx->cap_cl) {
    int** ip[] = {&ctx->d_cl_key, &ctx->d_cl_id, &ctx->d_cl_key2, &ctx->d_cl_id2};
    for (auto p : ip) {
      cudaFree(*p);
      *p = nullptr;
    }
    cudaFree(ctx->d_cl_f);
    cudaFree(ctx->d_cl_d);
    ctx->d_cl_f = nullptr;
    ctx->d_cl_d = nullptr;
    size_t c = 0;
    for (auto p : ip) {
      c = 0;
      SPS_TRY(sps_grow(ctx, p, c, (size_t)n));
    }
    c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_cl_f, c, (size_t)n));
    c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_cl_d, c, (size_t)n));
    ctx->cap_cl = n;
  }
  if ((size_t)ncells + 1 > ctx->cap_cl_cells) {
    cudaFree(ctx->d_cl_range);
    ctx->d_cl_range = nullptr;
    size_t c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_cl_range, c, (size_t)ncells + 1));
    ctx->cap_cl_cells = c;
  }
  k_cl_keys<<<nblk(n), kThreads, 0, ctx->stream>>>(n, pos, G, ctx->d_cl_key, ctx->d_cl_id);
  SPS_LAUNCHED(ctx);
  // counting sort by cell: histogram, exclusive scan (the per-cell ranges), scatter
  SPS_TRY(sps_grow(ctx, &ctx->d_cl_fill, ctx->cap_cl_fill, (size_t)ncells + 1));
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_cl_fill, 0, sizeof(int) * ((size_t)ncells + 1), ctx->stream));
  k_cell_hist<<<nblk(n), kThreads, 0, ctx->stream>>>(n, ctx->d_cl_key, ctx->d_cl_fill);
  SPS_LAUNCHED(ctx);
  SPS_TRY(exclusive_scan_impl(ctx, ctx->d_cl_fill, ctx->d_cl_range, (long long)ncells + 1));
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_cl_fill, 0, sizeof(int) * ((size_t)ncells + 1), ctx->stream));
  k_cell_scatter<<<nblk(n), kThreads, 0, ctx->stream>>>(n, ctx->d_cl_key, ctx->d_cl_id, ctx->d_cl_range,
                                                         ctx->d_cl_fill, ctx->d_cl_key2, ctx->d_cl_id2);
  SPS_LAUNCHED(ctx);
  k_cl_gather<<<nblk(n), kThreads, 0, ctx->stream>>>(n, ctx->d_cl_id2, pos, radii, G, ctx->d_cl_f,
                                                      ctx->d_cl_d);
  SPS_LAUNCHED(ctx);
  k_cl_count<<<nblk(n), kThreads, 0, ctx->stream>>>(n, ctx->d_cl_key2, ctx->d_cl_id2, ctx->d_cl_f,
                                                     ctx->d_cl_d, ctx->d_cl_range, G, acs, delta, drel,
                                                     ctx->d_ccount, ctx->d_ccount2);
  SPS_LAUNCHED(ctx);
  *Gout = G;
  *ncells_out = ncells;
  return SPS_OK;
}

}  // namespace

int sps_exclusive_scan(sps_ctx* ctx, const int* in, int* out, long long n) {
  return exclusive_scan_impl(ctx, in, out, n);
}

int sps_launch_contacts(sps_ctx* ctx, int n, const double* pos, const double* radii) {
  SpsPhase timer(ctx, SPS_PH_CONTACT);
  ctx->order_valid = false;
  const double acs = ctx->prm.a_c_scale, delta = ctx->prm.delta, drel = ctx->prm.delta_rel;
  const int search = ctx->prm.contact_search;
  const bool cells = search == SPS_SEARCH_CELLS || (search == SPS_SEARCH_AUTO && n > 4096);
  if ((size_t)n + 1 > ctx->cap_cnt) {
    int** ip[] = {&ctx->d_ccount, &ctx->d_ccount2, &ctx->d_inc_cnt, &ctx->d_cptr, &ctx->d_inc_ptr};
    for (auto p : ip) {
      cudaFree(*p);
      *p = nullptr;
    }
    size_t c = 0;
    for (auto p : ip) {
      c = 0;
      SPS_TRY(sps_grow(ctx, p, c, (size_t)n + 1));
    }
    ctx->cap_cnt = (size_t)n + 1;
  }
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_ccount, 0, sizeof(int) * (n + 1), ctx->stream));
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_ccount2, 0, sizeof(int) * (n + 1), ctx->stream));
  CellGrid G;
  int ncells = 0;
  if (cells) {
    SPS_TRY(cell_counts(ctx, n, pos, radii, &G, &ncells));
  } else {
    k_pairs_count<<<nblk(n, 128), 128, 0, ctx->stream>>>(n, pos, radii, acs, delta, drel, ctx->d_ccount,
                                                         ctx->d_ccount2);
    SPS_LAUNCHED(ctx);
  }
  k_add_counts<<<nblk(n + 1), kThreads, 0, ctx->stream>>>(n + 1, ctx->d_ccount, ctx->d_ccount2,
                                                          ctx->d_inc_cnt);
  SPS_LAUNCHED(ctx);
  const bool walls = ctx->walls.n > 0;
  if (walls) {
    SPS_TRY(sps_grow(ctx, &ctx->d_wcount, ctx->cap_wcount, (size_t)n + 1));
    SPS_TRY(sps_grow(ctx, &ctx->d_wptr, ctx->cap_wptr, (size_t)n + 1));
    k_wall_count<<<nblk(n + 1), kThreads, 0, ctx->stream>>>(n, pos, radii, ctx->walls, acs, delta, drel,
                                                            ctx->d_wcount, ctx->d_inc_cnt);
    SPS_LAUNCHED(ctx);
  }
  SPS_TRY(sps_exclusive_scan(ctx, ctx->d_ccount, ctx->d_cptr, n + 1));
  SPS_TRY(sps_exclusive_scan(ctx, ctx->d_inc_cnt, ctx->d_inc_ptr, n + 1));
  if (walls) SPS_TRY(sps_exclusive_scan(ctx, ctx->d_wcount, ctx->d_wptr, n + 1));
  int npair = 0, nwall = 0;
  SPS_TRY(read_int(ctx, ctx->d_cptr + n, &npair));
  if (walls) SPS_TRY(read_int(ctx, ctx->d_wptr + n, &nwall));
  const int nc = npair + nwall;
  ctx->n_c = nc;
  ctx->n_pair = npair;
  if (nc > ctx->cap_c) {
    int** ip[] = {&ctx->d_cij, &ctx->d_inc};
    for (auto p : ip) {
      cudaFree(*p);
      *p = nullptr;
    }
    cudaFree(ctx->d_cphi);
    cudaFree(ctx->d_cn);
    ctx->d_cphi = ctx->d_cn = nullptr;
    size_t c = 0;
    for (auto p : ip) {
      c = 0;
      SPS_TRY(sps_grow(ctx, p, c, 2 * (size_t)nc));
    }
    c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_cphi, c, (size_t)nc));
    c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_cn, c, 3 * (size_t)nc));
    ctx->cap_c = nc;
  }
  if (nc == 0) return SPS_OK;
  if (npair > 0) {
    if (cells) {
      k_cl_fill<<<nblk(n), kThreads, 0, ctx->stream>>>(n, ctx->d_cl_key2, ctx->d_cl_id2, ctx->d_cl_f,
                                                        ctx->d_cl_d, ctx->d_cl_range, G, acs, delta, drel,
                                                        ctx->d_cptr, ctx->d_cij);
    } else {
      k_pairs_fill<<<nblk(n, 128), 128, 0, ctx->stream>>>(n, pos, radii, acs, delta, drel, ctx->d_cptr,
                                                          ctx->d_cij);
    }
    SPS_LAUNCHED(ctx);
    k_contact_geom<<<nblk(npair), kThreads, 0, ctx->stream>>>(npair, ctx->d_cij, pos, radii, acs,
                                                               ctx->d_cphi, ctx->d_cn);
    SPS_LAUNCHED(ctx);
  }
  if (nwall > 0) {
    k_wall_fill<<<nblk(n), kThreads, 0, ctx->stream>>>(n, pos, radii, ctx->walls, acs, delta, drel, ctx->d_wptr,
                                                       npair, ctx->d_cij, ctx->d_cphi, ctx->d_cn);
    SPS_LAUNCHED(ctx);
  }
  // incidence lists: each sphere's contact ends in contact order (a
  // deterministic transpose of the list)
  if (!walls) {
    SPS_TRY(sps_grow(ctx, &ctx->d_wptr, ctx->cap_wptr, (size_t)n + 1));   // read only for wall rows
  }
  SPS_TRY(sps_grow(ctx, &ctx->d_inc_fill, ctx->cap_inc_fill, (size_t)n + 1));
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_inc_fill, 0, sizeof(int) * ((size_t)n + 1), ctx->stream));
  k_inc_fill<<<nblk(nc), kThreads, 0, ctx->stream>>>(nc, npair, ctx->d_cij, ctx->d_cptr, ctx->d_ccount,
                                                      ctx->d_ccount2, ctx->d_wptr, ctx->d_inc_ptr,
                                                      ctx->d_inc_fill, ctx->d_inc);
  SPS_LAUNCHED(ctx);
  k_inc_sort<<<nblk(n), kThreads, 0, ctx->stream>>>(n, ctx->d_inc_ptr, ctx->d_ccount2, ctx->d_inc);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_D(sps_ctx* ctx, const double* gamma, double* FT) {
  SpsPhase timer(ctx, SPS_PH_CONTACT);
  const int N = ctx->c_N;
  k_D<<<nblk(N), kThreads, 0, ctx->stream>>>(N, ctx->d_inc_ptr, ctx->d_inc, ctx->d_cn, gamma, FT);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_DT(sps_ctx* ctx, const double* UO, double* out) {
  SpsPhase timer(ctx, SPS_PH_CONTACT);
  if (ctx->n_c == 0) return SPS_OK;
  k_DT<<<nblk(ctx->n_c), kThreads, 0, ctx->stream>>>(ctx->n_c, ctx->d_cij, ctx->d_cn, UO, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// partials (5 x kStatBlocks) followed by the five results
static int ensure_bbpart(sps_ctx* ctx) {
  if (ctx->d_bbpart) return SPS_OK;
  size_t c = 0;
  return sps_grow(ctx, &ctx->d_bbpart, c, (size_t)5 * kStatBlocks + 8);
}

const double* sps_bb_out(sps_ctx* ctx) { return ctx->d_bbpart + 5 * kStatBlocks; }

int sps_bb_stats_dev(sps_ctx* ctx, const double* gn, const double* ggn, const double* go,
                     const double* ggo) {
  SpsPhase timer(ctx, SPS_PH_BBPGD);
  SPS_TRY(ensure_bbpart(ctx));
  const int nb = std::max(1, std::min(kStatBlocks, nblk(ctx->n_c)));
  k_bb_stats_part<<<nb, kThreads, 0, ctx->stream>>>(ctx->n_c, gn, ggn, go, ggo, ctx->d_bbpart);
  SPS_LAUNCHED(ctx);
  k_stat_finish<<<1, 160, 0, ctx->stream>>>(nb, ctx->d_bbpart, ctx->d_bbpart + 5 * kStatBlocks);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_bb_identity(sps_ctx* ctx, double alpha, const double* gam, const double* g,
                           double* gam_new, double* g_new) {
  SPS_TRY(ensure_bbpart(ctx));
  const int N = ctx->c_N, nc = ctx->n_c;
  {
    SpsPhase timer(ctx, SPS_PH_BBPGD);
    k_bb_proj<<<nblk(nc), kThreads, 0, ctx->stream>>>(nc, alpha, gam, g, gam_new);
    SPS_LAUNCHED(ctx);
  }
  {
    SpsPhase timer(ctx, SPS_PH_BB_D);
    if (!ctx->order_valid) {
      SPS_TRY(sps_grow(ctx, &ctx->d_order, ctx->cap_order, (size_t)N));
      k_degree_order<<<nblk(N), kThreads, 0, ctx->stream>>>(N, ctx->d_inc_ptr, ctx->d_order);
      SPS_LAUNCHED(ctx);
      ctx->order_valid = true;
    }
    k_bb_gather<<<nblk(N), kThreads, 0, ctx->stream>>>(N, ctx->d_order, ctx->d_inc_ptr, ctx->d_inc,
                                                        ctx->d_cn, gam_new, ctx->d_F3);
    SPS_LAUNCHED(ctx);
  }
  const int nb = std::max(1, std::min(kStatBlocks, nblk(nc)));
  {
    SpsPhase timer(ctx, SPS_PH_BB_DT);
    k_bb_ident_DT<<<nb, kThreads, 0, ctx->stream>>>(nc, ctx->d_cij, ctx->d_cn, ctx->d_F3, ctx->d_q,
                                                    gam_new, gam, g, ctx->prm.bb_variant != 1, g_new,
                                                    ctx->d_bbpart);
    SPS_LAUNCHED(ctx);
  }
  SpsPhase timer(ctx, SPS_PH_BBPGD);
  k_stat_finish<<<1, 160, 0, ctx->stream>>>(nb, ctx->d_bbpart, ctx->d_bbpart + 5 * kStatBlocks);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_identity_U(sps_ctx* ctx, int n, const double* FT, const double* F3, double* UO) {
  SpsPhase timer(ctx, SPS_PH_BBPGD);
  k_identity_U<<<nblk(6LL * n), kThreads, 0, ctx->stream>>>(n, FT, F3, UO);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_check_inputs(sps_ctx* ctx, int n, const double* pos, const double* radii, const double* FT) {
  if (!ctx->d_flag) {
    size_t c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_flag, c, 4));
  }
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  k_check<<<std::max(1, std::min(4 * 152, nblk(n))), kThreads, 0, ctx->stream>>>(n, pos, radii, FT,
                                                                                  ctx->d_flag);
  SPS_LAUNCHED(ctx);
  int f = 0;
  SPS_TRY(read_int(ctx, ctx->d_flag, &f));
  if (f & 1) return sps_fail(ctx, SPS_ERR_NONFINITE, "positions or radii not finite");
  if (f & 2) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "radii must be positive");
  if (f & 4) return sps_fail(ctx, SPS_ERR_NONFINITE, "force/torque not finite");
  return SPS_OK;
}

int sps_count_positive(sps_ctx* ctx, const double* v, int n, int* out) {
  if (!ctx->d_flag) {
    size_t c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_flag, c, 4));
  }
  *out = 0;
  if (n <= 0) return SPS_OK;
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  k_count_pos<<<std::max(1, std::min(4 * 152, nblk(n))), kThreads, 0, ctx->stream>>>(n, v, ctx->d_flag);
  SPS_LAUNCHED(ctx);
  return read_int(ctx, ctx->d_flag, out);
}

int sps_launch_contact_grad(sps_ctx* ctx, const double* pos, const double* mu, const double* w,
                            const double* U, double dt, double* dx) {
  SpsPhase timer(ctx, SPS_PH_CONTACT);
  const int N = ctx->c_N;
  if (ctx->n_c == 0) return SPS_OK;
  k_contact_grad<<<nblk(N), kThreads, 0, ctx->stream>>>(N, ctx->d_inc_ptr, ctx->d_inc, ctx->d_cij, ctx->d_cn,
                                                         pos, ctx->d_gam, mu, w, U, 1.0 / dt, dx);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}
