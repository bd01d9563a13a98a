// Geometry kernels: surface nodes (Sec. 5.4), near-pair lists (Sec. 4.2),
// rho from force/torque, the local operator L and velocity extraction
// (Sec. 4.1), and the contact builder that keeps its scratch in a static
// device array.  The contact search and D products are in sps_contacts.cu.

#include <mutex>

#include "sps_internal.cuh"

namespace {

constexpr int kThreads = 256;

inline int nblk(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// nodes: x = c + a n_k, normals n_k, weights a^2 w_k (Sec. 5.4)
// ---------------------------------------------------------------------------
// With rot (N x 9), node k of sphere s sits at c + a Q_s n_k, normal Q_s n_k.
__global__ void k_grid(int N, int P, const double* __restrict__ pos, const double* __restrict__ rad,
                       const double* __restrict__ un, const double* __restrict__ uw,
                       const double* __restrict__ rot,
                       double* __restrict__ X, double* __restrict__ Nr, double* __restrict__ W,
                       float* __restrict__ rel32, float* __restrict__ N32, float* __restrict__ W32,
                       float* __restrict__ chi, float* __restrict__ clo) {
  const long long NP = (long long)N * P;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NP;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / P), k = (int)(g - (long long)s * P);
    const double a = rad[s];
    double nv[3] = {un[k], un[P + k], un[2 * P + k]};
    if (rot) sps_rot_n(rot + 9 * s, nv[0], nv[1], nv[2]);
    for (int c = 0; c < 3; ++c) {
      const double n = nv[c];
      const double x = pos[3 * s + c] + a * n;
      X[c * NP + g] = x;
      Nr[c * NP + g] = n;
      rel32[c * NP + g] = (float)(a * n);     // offset from the sphere's centre
      N32[c * NP + g] = (float)n;
      if (k == 0) {                           // centre as an FP32 pair hi + lo
        const float hi = (float)pos[3 * s + c];
        chi[3 * s + c] = hi;
        clo[3 * s + c] = (float)(pos[3 * s + c] - (double)hi);
      }
    }
    const double w = a * a * uw[k];
    W[g] = w;
    W32[g] = (float)w;
  }
}

// near pairs: |c_i - c_j| < beta (a_i + a_j), j != i; sorted by j per i
__device__ __forceinline__ bool is_near(const double* pos, const double* rad, int i, int j,
                                        double beta) {
  const double dx = __dsub_rn(pos[3 * j + 0], pos[3 * i + 0]);
  const double dy = __dsub_rn(pos[3 * j + 1], pos[3 * i + 1]);
  const double dz = __dsub_rn(pos[3 * j + 2], pos[3 * i + 2]);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return sqrt(d2) < __dmul_rn(beta, __dadd_rn(rad[j], rad[i]));
}

__global__ void k_near_count(int N, const double* pos, const double* rad, double beta, int* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c = 0;
  for (int j = 0; j < N; ++j)
    if (j != i && is_near(pos, rad, i, j, beta)) ++c;
  cnt[i] = c;
}

__global__ void k_near_fill(int N, const double* pos, const double* rad, double beta,
                            const int* ptr, int* idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int o = ptr[i];
  for (int j = 0; j < N; ++j)
    if (j != i && is_near(pos, rad, i, j, beta)) idx[o++] = j;
}

// close near entries: node g of sphere i and near source j with
// |x_g - c_j| < kCloseRadius a_j
__global__ void k_close_count(int N, int P, const double* __restrict__ pos, const double* __restrict__ rad,
                              const double* __restrict__ X, const int* __restrict__ near_ptr,
                              const int* __restrict__ near_idx, int* __restrict__ cnt,
                              int* __restrict__ flag) {
  const long long NP = (long long)N * P;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g > NP) return;
  if (g == NP) {
    cnt[g] = 0;
    flag[g] = 0;
    return;
  }
  const int i = (int)(g / P);
  const double gx = X[g], gy = X[NP + g], gz = X[2 * NP + g];
  const double lim = sps::kCloseRadius * sps::kCloseRadius;
  int c = 0;
  for (int q = near_ptr[i]; q < near_ptr[i + 1]; ++q) {
    const int j = near_idx[q];
    if (sps_close_r2(pos, 1.0 / rad[j], gx, gy, gz, j) < lim) ++c;
  }
  cnt[g] = c;
  flag[g] = c > 0 ? 1 : 0;
}

__global__ void k_close_fill(int N, int P, const double* __restrict__ pos, const double* __restrict__ rad,
                             const double* __restrict__ X, const int* __restrict__ near_ptr,
                             const int* __restrict__ near_idx, const int* __restrict__ cnt,
                             const int* __restrict__ sptr, const int* __restrict__ fpos,
                             int* __restrict__ cnode, int* __restrict__ cptr, int* __restrict__ csrc) {
  const long long NP = (long long)N * P;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= NP || cnt[g] == 0) return;
  const int t = fpos[g];
  cnode[t] = (int)g;
  cptr[t] = sptr[g];
  cptr[t + 1] = sptr[g] + cnt[g];
  const int i = (int)(g / P);
  const double gx = X[g], gy = X[NP + g], gz = X[2 * NP + g];
  const double lim = sps::kCloseRadius * sps::kCloseRadius;
  int o = sptr[g];
  for (int q = near_ptr[i]; q < near_ptr[i + 1]; ++q) {
    const int j = near_idx[q];
    if (sps_close_r2(pos, 1.0 / rad[j], gx, gy, gz, j) < lim) csrc[o++] = j;
  }
}

// ---------------------------------------------------------------------------
// contacts (Sec. 3.2): i < j, Phi = (d - R_i) - R_j <= delta; every operation
// rounded separately so the list is reproducible to the bit.
// ---------------------------------------------------------------------------
using ContactGeom = SpsContactGeom;

__device__ __forceinline__ bool contact(const double* pos, const double* rad, double acs,
                                        double delta, int i, int j, ContactGeom* g) {
  return sps_contact_test(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], rad[i], pos[3 * j],
                          pos[3 * j + 1], pos[3 * j + 2], rad[j], acs, delta, 0.0, g);
}

// rho = F/|Gamma| + tau^{-1} T x (x - c), tau = (8 pi/3) a^4 (Sec. 4.1)
__global__ void k_rho(int N, int P, const double* __restrict__ pos, const double* __restrict__ rad,
                      const double* __restrict__ X, const double* __restrict__ FT,
                      double* __restrict__ rho) {
  const long long NP = (long long)N * P;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NP;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / P);
    const double a = rad[s];
    const double ia = 1.0 / (4.0 * SPS_PI * a * a), it = 3.0 / (8.0 * SPS_PI * a * a * a * a);
    const double rx = X[g] - pos[3 * s], ry = X[NP + g] - pos[3 * s + 1],
                 rz = X[2 * NP + g] - pos[3 * s + 2];
    const double* T = FT + 6 * s + 3;
    rho[g] = FT[6 * s + 0] * ia + it * (T[1] * rz - T[2] * ry);
    rho[NP + g] = FT[6 * s + 1] * ia + it * (T[2] * rx - T[0] * rz);
    rho[2 * NP + g] = FT[6 * s + 2] * ia + it * (T[0] * ry - T[1] * rx);
  }
}

// per sphere: int f dS and int (x - c) x f dS (one warp per sphere)
__global__ void k_moments(int N, int P, const double* __restrict__ pos, const double* __restrict__ X,
                          const double* __restrict__ W, const double* __restrict__ f,
                          double* __restrict__ mom) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  const long long NP = (long long)N * P;
  const int s = warp;
  double m[6] = {0, 0, 0, 0, 0, 0};
  for (int k = lane; k < P; k += 32) {
    const long long g = (long long)s * P + k;
    const double w = W ? W[g] : 1.0;
    const double fx = f[g] * w, fy = f[NP + g] * w, fz = f[2 * NP + g] * w;
    const double rx = X[g] - pos[3 * s], ry = X[NP + g] - pos[3 * s + 1],
                 rz = X[2 * NP + g] - pos[3 * s + 2];
    m[0] += fx;
    m[1] += fy;
    m[2] += fz;
    m[3] += ry * fz - rz * fy;
    m[4] += rz * fx - rx * fz;
    m[5] += rx * fy - ry * fx;
  }
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) m[c] += __shfl_xor_sync(0xffffffffu, m[c], o);
  if (lane == 0)
    for (int c = 0; c < 6; ++c) mom[6 * s + c] = m[c];
}

// out += L[f]: f-moments per sphere broadcast back (Sec. 4.1, operator L)
__global__ void k_add_L(int N, int P, const double* __restrict__ pos, const double* __restrict__ rad,
                        const double* __restrict__ X, const double* __restrict__ mom,
                        const double* __restrict__ Wout, double* __restrict__ out) {
  const long long NP = (long long)N * P;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NP;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / P);
    const double a = rad[s];
    const double ia = 1.0 / (4.0 * SPS_PI * a * a), it = 3.0 / (8.0 * SPS_PI * a * a * a * a);
    const double rx = X[g] - pos[3 * s], ry = X[NP + g] - pos[3 * s + 1],
                 rz = X[2 * NP + g] - pos[3 * s + 2];
    const double* m = mom + 6 * s;
    const double tx = it * m[3], ty = it * m[4], tz = it * m[5];
    const double wo = Wout ? Wout[g] : 1.0;
    out[g] += wo * (m[0] * ia + (ty * rz - tz * ry));
    out[NP + g] += wo * (m[1] * ia + (tz * rx - tx * rz));
    out[2 * NP + g] += wo * (m[2] * ia + (tx * ry - ty * rx));
  }
}

__global__ void k_extract(int N, const double* __restrict__ rad, const double* __restrict__ mom,
                          double* __restrict__ UO) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const double a = rad[s];
  const double ia = 1.0 / (4.0 * SPS_PI * a * a), it = 3.0 / (8.0 * SPS_PI * a * a * a * a);
  for (int c = 0; c < 3; ++c) {
    UO[6 * s + c] = mom[6 * s + c] * ia;
    UO[6 * s + 3 + c] = mom[6 * s + 3 + c] * it;
  }
}

}  // namespace

int sps_launch_grid(sps_ctx* ctx) {
  SpsPhase timer(ctx, SPS_PH_GEOM);
  const long long NP = ctx->NP;
  k_grid<<<nblk(NP), kThreads, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos, ctx->d_rad,
                                                  ctx->d_unit_nrm, ctx->d_unit_w,
                                                  ctx->rot_n == ctx->N ? ctx->d_rot : nullptr, ctx->d_X,
                                                  ctx->d_Nrm, ctx->d_W, ctx->d_rel32, ctx->d_N32,
                                                  ctx->d_W32, ctx->d_chi, ctx->d_clo);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

namespace {
__global__ void k_rotate(int N, int P, const double* __restrict__ rot, const double* in, double* out,
                         int transpose) {
  const long long NP = (long long)N * P;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NP;
       g += (long long)gridDim.x * blockDim.x) {
    const double* Q = rot + 9 * (g / P);
    double x = in[g], y = in[NP + g], z = in[2 * NP + g];
    if (transpose)
      sps_rot_t(Q, x, y, z);
    else
      sps_rot_n(Q, x, y, z);
    out[g] = x;
    out[NP + g] = y;
    out[2 * NP + g] = z;
  }
}
}  // namespace

int sps_launch_rotate(sps_ctx* ctx, const double* in, double* out, bool transpose) {
  SpsPhase timer(ctx, SPS_PH_SELF);
  k_rotate<<<(int)std::min<long long>(nblk(ctx->NP), 8 * 152), kThreads, 0, ctx->stream>>>(
      ctx->N, ctx->T.P, ctx->d_rot, in, out, transpose ? 1 : 0);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_near_lists(sps_ctx* ctx) {
  SpsPhase timer(ctx, SPS_PH_GEOM);
  const int N = ctx->N;
  size_t cap = 0;
  int* d_cnt = nullptr;
  SPS_TRY(sps_grow(ctx, &d_cnt, cap, (size_t)N + 1));
  k_near_count<<<nblk(N, 128), 128, 0, ctx->stream>>>(N, ctx->d_pos, ctx->d_rad, ctx->prm.beta, d_cnt);
  SPS_LAUNCHED(ctx);
  // exclusive scan into near_ptr (N+1)
  SPS_CUDA(ctx, cudaMemsetAsync(d_cnt + N, 0, sizeof(int), ctx->stream));
  SPS_TRY(sps_exclusive_scan(ctx, d_cnt, ctx->d_near_ptr, N + 1));
  int total = 0;
  SPS_CUDA(ctx, cudaMemcpyAsync(&total, ctx->d_near_ptr + N, sizeof(int), cudaMemcpyDeviceToHost,
                                ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  cudaFree(d_cnt);
  size_t capn = ctx->cap_near;
  SPS_TRY(sps_grow(ctx, &ctx->d_near_idx, capn, (size_t)total));
  ctx->cap_near = (int)capn;
  ctx->n_near = total;
  k_near_fill<<<nblk(N, 128), 128, 0, ctx->stream>>>(N, ctx->d_pos, ctx->d_rad, ctx->prm.beta,
                                                      ctx->d_near_ptr, ctx->d_near_idx);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

namespace {
// For each position q' of the near CSR (row j, source-major reading: target
// i = near_idx[q'] of source j): rev[q'] = the position q of j in row i (the
// relation is symmetric to the bit), and geo[q'] = (c_j - c_i) / a_i, the
// offset of sphere j's centre seen from near source i in i's radius units
// (FP32), which the source-major near field reads through rev.
__global__ void k_near_rev(int N, const int* __restrict__ ptr, const int* __restrict__ idx,
                           const double* __restrict__ pos, const double* __restrict__ rad,
                           int* __restrict__ rev, float* __restrict__ geo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  for (int qp = ptr[j]; qp < ptr[j + 1]; ++qp) {
    const int i = idx[qp];
    int lo = ptr[i], hi = ptr[i + 1] - 1, q = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1, v = idx[mid];
      if (v == j) {
        q = mid;
        break;
      }
      if (v < j) lo = mid + 1;
      else hi = mid - 1;
    }
    rev[qp] = q;
    const double ia = 1.0 / rad[i];
    geo[3 * qp] = (float)((pos[3 * j] - pos[3 * i]) * ia);
    geo[3 * qp + 1] = (float)((pos[3 * j + 1] - pos[3 * i + 1]) * ia);
    geo[3 * qp + 2] = (float)((pos[3 * j + 2] - pos[3 * i + 2]) * ia);
  }
}
}  // namespace

int sps_launch_near_rev(sps_ctx* ctx) {
  SpsPhase timer(ctx, SPS_PH_GEOM);
  const size_t nq = (size_t)std::max(ctx->n_near, 1);
  SPS_TRY(sps_grow(ctx, &ctx->d_near_rev, ctx->cap_near_rev, nq));
  SPS_TRY(sps_grow(ctx, &ctx->d_near_geo, ctx->cap_near_geo, 3 * nq));
  if (ctx->n_near == 0) return SPS_OK;
  k_near_rev<<<nblk(ctx->N, 128), 128, 0, ctx->stream>>>(ctx->N, ctx->d_near_ptr, ctx->d_near_idx, ctx->d_pos,
                                                          ctx->d_rad, ctx->d_near_rev, ctx->d_near_geo);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_close_lists(sps_ctx* ctx) {
  SpsPhase timer(ctx, SPS_PH_GEOM);
  const long long NP = ctx->NP;
  int *d_cnt = nullptr, *d_flag = nullptr, *d_sptr = nullptr, *d_fpos = nullptr;
  size_t c1 = 0, c2 = 0, c3 = 0, c4 = 0;
  SPS_TRY(sps_grow(ctx, &d_cnt, c1, (size_t)NP + 1));
  SPS_TRY(sps_grow(ctx, &d_flag, c2, (size_t)NP + 1));
  SPS_TRY(sps_grow(ctx, &d_sptr, c3, (size_t)NP + 1));
  SPS_TRY(sps_grow(ctx, &d_fpos, c4, (size_t)NP + 1));
  k_close_count<<<nblk(NP + 1), kThreads, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos, ctx->d_rad,
                                                             ctx->d_X, ctx->d_near_ptr, ctx->d_near_idx,
                                                             d_cnt, d_flag);
  SPS_LAUNCHED(ctx);
  SPS_TRY(sps_exclusive_scan(ctx, d_cnt, d_sptr, NP + 1));
  SPS_TRY(sps_exclusive_scan(ctx, d_flag, d_fpos, NP + 1));
  int tot[2] = {0, 0};
  SPS_CUDA(ctx, cudaMemcpyAsync(&tot[0], d_fpos + NP, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA(ctx, cudaMemcpyAsync(&tot[1], d_sptr + NP, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->n_close = tot[0];
  ctx->n_close_src = tot[1];
  SPS_TRY(sps_grow(ctx, &ctx->d_close_node, ctx->cap_close_node, (size_t)tot[0] + 1));
  SPS_TRY(sps_grow(ctx, &ctx->d_close_ptr, ctx->cap_close_ptr, (size_t)tot[0] + 2));
  SPS_TRY(sps_grow(ctx, &ctx->d_close_src, ctx->cap_close_src, (size_t)tot[1] + 1));
  if (tot[0] > 0) {
    k_close_fill<<<nblk(NP), kThreads, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos, ctx->d_rad, ctx->d_X,
                                                          ctx->d_near_ptr, ctx->d_near_idx, d_cnt, d_sptr,
                                                          d_fpos, ctx->d_close_node, ctx->d_close_ptr,
                                                          ctx->d_close_src);
    SPS_LAUNCHED(ctx);
  }
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  cudaFree(d_cnt);
  cudaFree(d_flag);
  cudaFree(d_sptr);
  cudaFree(d_fpos);
  return SPS_OK;
}

int sps_launch_rho(sps_ctx* ctx, const double* FT, double* rho) {
  SpsPhase timer(ctx, SPS_PH_KRYLOV);
  k_rho<<<nblk(ctx->NP), kThreads, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos, ctx->d_rad,
                                                      ctx->d_X, FT, rho);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_moments(sps_ctx* ctx, const double* f, double* mom) {
  SpsPhase timer(ctx, SPS_PH_KRYLOV);
  k_moments<<<nblk((long long)ctx->N * 32, 128), 128, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos,
                                                                        ctx->d_X, ctx->d_W, f, mom);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_add_L(sps_ctx* ctx, const double* mom, double* out) {
  SpsPhase timer(ctx, SPS_PH_KRYLOV);
  k_add_L<<<nblk(ctx->NP), kThreads, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos, ctx->d_rad,
                                                        ctx->d_X, mom, nullptr, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_add_L_w(sps_ctx* ctx, const double* mom, double* out, bool weight_out) {
  SpsPhase timer(ctx, SPS_PH_KRYLOV);
  k_add_L<<<nblk(ctx->NP), kThreads, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos, ctx->d_rad,
                                                        ctx->d_X, mom, weight_out ? ctx->d_W : nullptr, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_moments_w(sps_ctx* ctx, const double* f, double* mom, bool weighted) {
  SpsPhase timer(ctx, SPS_PH_KRYLOV);
  k_moments<<<nblk((long long)ctx->N * 32, 128), 128, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_pos,
                                                                        ctx->d_X, weighted ? ctx->d_W : nullptr,
                                                                        f, mom);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_extract(sps_ctx* ctx, const double* mom, double* UO) {
  SpsPhase timer(ctx, SPS_PH_KRYLOV);
  k_extract<<<nblk(ctx->N), kThreads, 0, ctx->stream>>>(ctx->N, ctx->d_rad, mom, UO);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// ---------------------------------------------------------------------------
// Contact set without allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// contact list: code embedded in a host whose own memory pool has reserved the
// device (a framework's caching allocator, an MPS client with a hard memory
// limit), where a cudaMalloc outside that pool fails or fragments it, or a
// time-stepping loop that must not pay for, or risk failing on, an allocation
// in the middle of a step.  This variant of the contact builder keeps its only
// scratch (one counter per sphere plus the scan's block totals) in a fixed
// device array that lives as long as the library is loaded.  The caller passes
// positions, radii and output buffers.  It searches all pairs (one thread per
// sphere i over j > i), O(n^2) pair tests, with the absolute threshold delta
// only (no relative part).
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxSpheres = 1 << 18;     // 262,144 spheres
constexpr int kScanThreads = 1024;
// counters (max spheres + 1) followed by one total per scan thread
static __device__ __align__(256) int g_contact_scratch[kStaticMaxSpheres + 1 + kScanThreads];

__global__ void k_static_count(int N, const double* pos, const double* rad, double acs, double delta,
                               int* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) cnt[N] = 0;   // the scan's last slot (the total) starts at zero
  if (i >= N) return;
  int c = 0;
  for (int j = i + 1; j < N; ++j)
    if (contact(pos, rad, acs, delta, i, j, nullptr)) ++c;
  cnt[i] = c;
}

// exclusive scan of cnt[0..n) in place, one block; totals[] holds per-thread sums
__global__ void __launch_bounds__(kScanThreads) k_static_scan(int n, int* cnt, int* totals) {
  const int t = threadIdx.x;
  const int per = (n + kScanThreads - 1) / kScanThreads;
  const int a = min(n, t * per), b = min(n, a + per);
  int s = 0;
  for (int i = a; i < b; ++i) s += cnt[i];
  totals[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int k = 0; k < kScanThreads; ++k) {
      const int v = totals[k];
      totals[k] = run;
      run += v;
    }
  }
  __syncthreads();
  int run = totals[t];
  for (int i = a; i < b; ++i) {
    const int v = cnt[i];
    cnt[i] = run;
    run += v;
  }
}

__global__ void k_static_fill(int N, const double* pos, const double* rad, double acs, double delta,
                              const int* ptr, int* ij, double* phi, double* nrm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int o = ptr[i];
  ContactGeom g;
  for (int j = i + 1; j < N; ++j)
    if (contact(pos, rad, acs, delta, i, j, &g)) {
      ij[2 * o] = i;
      ij[2 * o + 1] = j;
      phi[o] = g.phi;
      nrm[3 * o + 0] = g.nx;
      nrm[3 * o + 1] = g.ny;
      nrm[3 * o + 2] = g.nz;
      ++o;
    }
}

// Host-side stand-in for g_contact_scratch is not a device address: resolve
// the real address once per device, with that device current.
std::mutex g_scratch_mu;
int* g_scratch_ptr[64] = {nullptr};

int static_scratch(int** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return SPS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_contact_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SPS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<int*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SPS_OK;
}

}  // namespace

extern "C" int sps_build_contacts_noalloc(int n, const double* pos, const double* radii,
                                          double a_c_scale, double delta, int max_contacts, int* ij,
                                          double* phi, double* normals, int* n_contacts_out,
                                          void* stream) {
  if (n < 1 || !pos || !radii || !n_contacts_out || max_contacts < 0 || !(a_c_scale > 0) ||
      !(delta >= 0) || (max_contacts > 0 && (!ij || !phi || !normals)))
    return SPS_ERR_INVALID_ARG;
  if (n > kStaticMaxSpheres) return SPS_ERR_CAPACITY;
  int* cnt = nullptr;
  int rc = static_scratch(&cnt);
  if (rc != SPS_OK) return rc;
  int* totals = cnt + kStaticMaxSpheres + 1;
  cudaStream_t st = (cudaStream_t)stream;
  k_static_count<<<(n + 127) / 128, 128, 0, st>>>(n, pos, radii, a_c_scale, delta, cnt);
  if (cudaGetLastError() != cudaSuccess) return SPS_ERR_CUDA;
  k_static_scan<<<1, kScanThreads, 0, st>>>(n + 1, cnt, totals);
  if (cudaGetLastError() != cudaSuccess) return SPS_ERR_CUDA;
  int nc = 0;
  if (cudaMemcpyAsync(&nc, cnt + n, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_CUDA;
  }
  *n_contacts_out = nc;
  if (nc > max_contacts) return SPS_ERR_CAPACITY;
  if (nc > 0) {
    k_static_fill<<<(n + 127) / 128, 128, 0, st>>>(n, pos, radii, a_c_scale, delta, cnt, ij, phi,
                                                   normals);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return SPS_ERR_CUDA;
    }
  }
  return SPS_OK;
}
