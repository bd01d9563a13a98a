// Context, mobility solve and collision resolution (C ABI of include/sps.h).
//
//  * Mobility (Sec. 4.1): rho from F, T; GMRES on (I/2 + K + L)[mu] = L[rho]
//    for mu = rho + zeta (eq. rigidbodyrho rearranged: the same discrete
//    solution, no traction application on its right-hand side);
//    u = S[rho + zeta] = S[mu] (eq. velS); U, Omega as averages of u over
//    each sphere.
//    GMRES: unrestarted, zero or warm initial guess, classical Gram-Schmidt applied
//    twice, Givens rotations on the host, FP64 everywhere; stop when
//    ||r|| / ||b|| < gmres_tol.  Mixed precision: the far-field sums run in
//    FP32 (compensated), the Krylov basis, orthogonalisation and residual in
//    FP64; with ir_tol > 0 the solve is refined against the FP64 operator.
//  * Collision step (Sec. 3.2, Algorithm 1): contacts, q = Phi/dt + D^T U_nc,
//    BBPGD with gamma_0 = 0 (M gamma_0 = 0 needs no solve), alpha_0 =
//    g^T g / g^T M g, projected steps, min-map residual test, BB1 or BB2
//    step lengths; U = U_nc + M D gamma; pos += U dt.
//  All reductions are deterministic (fixed block partition and order).
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <vector>

#include "sps_internal.cuh"

namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;
constexpr int kChunk = 8;   // dot products per pass of the multi-dot kernel

// partial[j][b] = sum over block b's slice of Q_j . w for j < k, and
// partial[k][b] = the slice's w . w: every dot product of one Gram-Schmidt pass
// plus the squared norm in one launch (fixed slice partition: deterministic).
__global__ void __launch_bounds__(kRedThreads) k_multidot(long long n, const double* __restrict__ Q,
                                                         long long ldq, int k,
                                                         const double* __restrict__ w,
                                                         double* __restrict__ partial) {
  __shared__ double red[kRedThreads / 32][kChunk];
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long a = blockIdx.x * per, b = min(n, a + per);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j0 = 0; j0 <= k; j0 += kChunk) {
    const int nj = min(kChunk, k + 1 - j0);
    double acc[kChunk];
#pragma unroll
    for (int q = 0; q < kChunk; ++q) acc[q] = 0.0;
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int q = 0; q < kChunk; ++q) {
        const int j = j0 + q;
        if (q < nj) acc[q] = fma(j < k ? Q[(long long)j * ldq + i] : wi, wi, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < kChunk; ++q) red[warp][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < nj) {
      double s = 0.0;
      for (int v = 0; v < kRedThreads / 32; ++v) s += red[v][threadIdx.x];
      partial[(long long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
  }
}

__global__ void k_finish(int nj, int nb, const double* __restrict__ partial, double* __restrict__ h) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nj) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[(long long)j * nb + b];
  h[j] = s;
}

// w -= sum_j h_j Q_j   (h on device)
__global__ void k_sub_proj(long long n, const double* __restrict__ Q, long long ldq, int k,
                           const double* __restrict__ h, double* __restrict__ w) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int j = 0; j < k; ++j) s = fma(-h[j], Q[(long long)j * ldq + i], s);
    w[i] = s;
  }
}

// x = sum_j y_j Q_j (+ x if accumulate)
__global__ void k_combine(long long n, const double* __restrict__ Q, long long ldq, int k,
                          const double* __restrict__ y, int accumulate, double* __restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double s = accumulate ? x[i] : 0.0;
    for (int j = 0; j < k; ++j) s = fma(y[j], Q[(long long)j * ldq + i], s);
    x[i] = s;
  }
}

__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    z[i] = a * x[i] + b * (y ? y[i] : 0.0);
}

// BBPGD: gamma_new = max(gamma - alpha g, 0)
__global__ void k_bb_step(int n, double alpha, const double* __restrict__ gam,
                          const double* __restrict__ g, double* __restrict__ gnew) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) gnew[l] = fmax(gam[l] - alpha * g[l], 0.0);
}

// g = a + q
__global__ void k_add(int n, const double* __restrict__ a, const double* __restrict__ q,
                      double* __restrict__ g) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) g[l] = a[l] + q[l];
}

// gamma_0 for a new contact list from the previous step's solution: the
// value of the same pair (i, j) if it was a contact then, else 0 (both lists
// sorted by (i, j); binary search)
// gamma_0 from the previous step's list: sphere pairs are sorted by (i, j),
// wall contacts (first index -1 - w) after them by (sphere, wall); each block
// is searched on its own order
__global__ void k_map_gamma(int nc, const int* __restrict__ ij, int npair, int nprev, int nprev_pair,
                            const int* __restrict__ pij, const double* __restrict__ pgam,
                            double* __restrict__ gam) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nc) return;
  const int i = ij[2 * l], j = ij[2 * l + 1];
  const bool wall = l >= npair;
  // key (a, b): (i, j) for pairs, (sphere, wall) for walls
  const int a = wall ? j : i, b = wall ? -1 - i : j;
  int lo = wall ? nprev_pair : 0, hi = wall ? nprev : nprev_pair;
  const int end = hi;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int pa = wall ? pij[2 * mid + 1] : pij[2 * mid], pb = wall ? -1 - pij[2 * mid] : pij[2 * mid + 1];
    if (pa < a || (pa == a && pb < b)) lo = mid + 1;
    else hi = mid;
  }
  gam[l] = (lo < end && pij[2 * lo] == i && pij[2 * lo + 1] == j) ? pgam[lo] : 0.0;
}

// q = phi/dt + D^T U_nc (D^T U_nc already in q)
__global__ void k_q(int n, const double* __restrict__ phi, double idt, double* __restrict__ q) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) q[l] = phi[l] * idt + q[l];
}

__global__ void k_pos_update(int n, const double* __restrict__ pos, const double* __restrict__ UO,
                             double dt, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) out[i] = pos[i] + dt * UO[6 * (i / 3) + (i % 3)];
}

// rbar = sbar - (lam/2 + rbar): finishes rhobar = sbar - (I/2 + K)^T lambda
__global__ void k_combine3(long long n, const double* __restrict__ sbar, const double* __restrict__ lam,
                           double* __restrict__ rbar) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    rbar[i] = sbar[i] - (0.5 * lam[i] + rbar[i]);
}

inline int gblocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 8 * 152); }

}  // namespace

static cudaEvent_t pool_event(sps_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

SpsPhase::SpsPhase(sps_ctx* ctx, int phase) : c(ctx), ph(phase) {
  if (!c->prof) return;
  b = pool_event(c);
  e = pool_event(c);
  if (b) cudaEventRecord(b, c->stream);
}

SpsPhase::~SpsPhase() {
  if (!c->prof || !b || !e) return;
  cudaEventRecord(e, c->stream);
  c->ev_rec.push_back({ph, {b, e}});
}

extern "C" int sps_profile(sps_ctx* ctx, int enable) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->prof = enable != 0;
  ctx->ev_rec.clear();
  ctx->ev_used = 0;
  return SPS_OK;
}

extern "C" int sps_profile_read(sps_ctx* ctx, double* ms, long long* launches) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double t[SPS_PH_COUNT] = {0};
  long long n[SPS_PH_COUNT] = {0};
  for (auto& r : ctx->ev_rec) {
    float x = 0.f;
    SPS_CUDA(ctx, cudaEventElapsedTime(&x, r.second.first, r.second.second));
    t[r.first] += x;
    n[r.first] += 1;
  }
  if (ms) std::memcpy(ms, t, sizeof(t));
  if (launches) std::memcpy(launches, n, sizeof(n));
  return SPS_OK;
}

int sps_fail(sps_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

// out[0..k) = Q[0..k)^T w and out[k] = w . w, on the device (no sync)
// partial: (k + 1) x kRedBlocks doubles (the GMRES workspace, or d_sc for k = 1)
static int multidot_dev(sps_ctx* ctx, const double* Q, long long ldq, int k, const double* w,
                        long long n, double* out, double* partial) {
  { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
  k_multidot<<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(n, Q, ldq, k, w, partial); }
  SPS_LAUNCHED(ctx);
  { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
  k_finish<<<(k + 1 + 127) / 128, 128, 0, ctx->stream>>>(k + 1, kRedBlocks, partial, out); }
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

static int to_host(sps_ctx* ctx, const double* d, int cnt, double* h) {
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost,
                                ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::memcpy(h, ctx->h_pinned, sizeof(double) * cnt);
  return SPS_OK;
}

// a . b (host result); uses the multi-dot kernel with a one-vector "basis"
int sps_dot(sps_ctx* ctx, const double* a, const double* b, long long n, double* out) {
  // k = 1 with Q = a gives out[0] = a.b (out[1] = b.b is ignored)
  double* res = ctx->d_sc + 2 * kRedBlocks;
  SPS_TRY(multidot_dev(ctx, a, 0, 1, b, n, res, ctx->d_sc));
  double tmp[2];
  SPS_TRY(to_host(ctx, res, 2, tmp));
  *out = tmp[0];
  return SPS_OK;
}

static int ensure_gmres(sps_ctx* ctx, long long n, int kmax) {
  if (n <= ctx->gm_cap_n && kmax <= ctx->gm_cap_k && ctx->d_Q) return SPS_OK;
  cudaFree(ctx->d_Q);
  cudaFree(ctx->d_w);
  cudaFree(ctx->d_h);
  cudaFree(ctx->d_red);
  ctx->d_Q = ctx->d_w = ctx->d_h = ctx->d_red = nullptr;
  size_t c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_Q, c, (size_t)(kmax + 1) * n));
  c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_w, c, (size_t)n));
  c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_h, c, 2 * (size_t)kmax + 16));
  c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_red, c, (size_t)(kmax + 8) * kRedBlocks));
  ctx->gm_cap_n = (int)n;
  ctx->gm_cap_k = kmax;
  return SPS_OK;
}

// operator application for GMRES: out = (I/2 + K + L) v, or its transpose
// while an adjoint solve runs
static int apply_A(sps_ctx* ctx, const double* v, double* out, bool fp32) {
  if (ctx->adjoint_mode) return sps_layer_T(ctx, SPS_OP_A, v, out);
  return sps_layer(ctx, SPS_OP_A, v, out, fp32);
}

// GMRES on A x = b.  warm: x holds an initial guess (else x0 = 0); r0: its
// residual b - A x0 when the caller knows it (else one application of A).
// Stops when ||b - A x|| / ||b|| < tol.  Classical Gram-Schmidt applied twice;
// each Arnoldi step reads its dot products and norm back with one
// synchronisation: the norm after the second pass is sqrt(||w||^2 - ||h2||^2)
// (w is then orthogonal to the basis).  Ax (optional) receives A x from the
// Arnoldi relation, A x = b - r0 + V_{k+1} Hbar y, without applying A.
// Returns SPS_OK or NOT_CONVERGED.
static int gmres(sps_ctx* ctx, const double* b, double* x, bool warm, double tol, int kmax,
                 bool fp32, int* iters, double* relres, const double* r0 = nullptr,
                 double* Ax = nullptr) {
  const long long n = 3LL * ctx->NP;
  SPS_TRY(ensure_gmres(ctx, n, kmax));
  double bb = 0.0;
  SPS_TRY(sps_dot(ctx, b, b, n, &bb));
  if (!std::isfinite(bb)) return sps_fail(ctx, SPS_ERR_NONFINITE, "GMRES right-hand side is not finite");
  const double nb = std::sqrt(bb);
  *iters = 0;
  *relres = 0.0;
  if (nb == 0.0) {
    SPS_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
    if (Ax) SPS_CUDA(ctx, cudaMemsetAsync(Ax, 0, sizeof(double) * n, ctx->stream));
    return SPS_OK;
  }
  double* Q = ctx->d_Q;
  double* w = ctx->d_w;
  // r0 = b - A x0 (in Q_0 before normalisation)
  double beta = nb;
  if (warm) {
    if (r0) {
      SPS_CUDA(ctx, cudaMemcpyAsync(Q, r0, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
      SPS_TRY(apply_A(ctx, x, w, fp32));
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, 1.0, b, -1.0, w, Q); }
      SPS_LAUNCHED(ctx);
    }
    double rr = 0.0;
    SPS_TRY(sps_dot(ctx, Q, Q, n, &rr));
    if (std::isfinite(rr)) {
      beta = std::sqrt(rr);
      if (beta / nb < tol) {
        *relres = beta / nb;
        if (Ax) {
          SpsPhase timer_(ctx, SPS_PH_KRYLOV);
          k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, 1.0, b, -1.0, Q, Ax);
          SPS_LAUNCHED(ctx);
        }
        return SPS_OK;
      }
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, 1.0 / beta, Q, 0.0, nullptr, Q); }
      SPS_LAUNCHED(ctx);
    } else {
      // the guess is unusable (not finite): start from x0 = 0 instead
      warm = false;
      beta = nb;
      SPS_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
    }
  }
  if (!warm) {
    { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
    k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, 1.0 / beta, b, 0.0, nullptr, Q); }
    SPS_LAUNCHED(ctx);
  }
  std::vector<double> H((size_t)(kmax + 1) * kmax, 0.0), cs(kmax), sn(kmax), g(kmax + 1, 0.0);
  std::vector<double> Hbar(Ax ? (size_t)(kmax + 1) * kmax : 0);   // before the rotations
  std::vector<double> hh(2 * kmax + 4);
  g[0] = beta;
  int k = 0;
  double res = beta / nb;
  auto Hc = [&](int r, int c) -> double& { return H[(size_t)c * (kmax + 1) + r]; };
  double* d_h1 = ctx->d_h;
  double* d_h2 = ctx->d_h + kmax + 8;
  for (k = 1; k <= kmax; ++k) {
    SPS_TRY(apply_A(ctx, Q + (long long)(k - 1) * n, w, fp32));
    SPS_TRY(multidot_dev(ctx, Q, n, k, w, n, d_h1, ctx->d_red));
    { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
    k_sub_proj<<<gblocks(n), 256, 0, ctx->stream>>>(n, Q, n, k, d_h1, w); }
    SPS_LAUNCHED(ctx);
    SPS_TRY(multidot_dev(ctx, Q, n, k, w, n, d_h2, ctx->d_red));
    { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
    k_sub_proj<<<gblocks(n), 256, 0, ctx->stream>>>(n, Q, n, k, d_h2, w); }
    SPS_LAUNCHED(ctx);
    // one read-back: h1 (k), h2 (k) and ||w||^2 before the second projection
    SPS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, d_h1, sizeof(double) * k, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + k, d_h2, sizeof(double) * (k + 1),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::memcpy(hh.data(), ctx->h_pinned, sizeof(double) * (2 * k + 1));
    double h2sq = 0.0;
    for (int j = 0; j < k; ++j) h2sq += hh[k + j] * hh[k + j];
    const double ww = hh[2 * k] - h2sq;
    if (!std::isfinite(ww)) return sps_fail(ctx, SPS_ERR_NONFINITE, "GMRES: non-finite Krylov vector");
    const double hk = std::sqrt(std::max(ww, 0.0));
    for (int j = 0; j < k; ++j) Hc(j, k - 1) = hh[j] + hh[k + j];
    Hc(k, k - 1) = hk;
    if (Ax)
      std::copy(&Hc(0, k - 1), &Hc(0, k - 1) + k + 1, Hbar.begin() + (size_t)(k - 1) * (kmax + 1));
    if (hk > 0.0) {
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, 1.0 / hk, w, 0.0, nullptr, Q + (long long)k * n); }
      SPS_LAUNCHED(ctx);
    }
    for (int j = 0; j < k - 1; ++j) {
      const double a = Hc(j, k - 1), bq = Hc(j + 1, k - 1);
      Hc(j, k - 1) = cs[j] * a + sn[j] * bq;
      Hc(j + 1, k - 1) = -sn[j] * a + cs[j] * bq;
    }
    const double a = Hc(k - 1, k - 1), bq = Hc(k, k - 1);
    const double den = std::hypot(a, bq);
    if (!(den > 0.0)) {   // A q_{k-1} = 0 exactly: keep the first k-1 columns
      --k;
      break;
    }
    cs[k - 1] = a / den;
    sn[k - 1] = bq / den;
    Hc(k - 1, k - 1) = den;
    Hc(k, k - 1) = 0.0;
    g[k] = -sn[k - 1] * g[k - 1];
    g[k - 1] = cs[k - 1] * g[k - 1];
    res = std::fabs(g[k]) / nb;
    if (res < tol || hk == 0.0) break;
  }
  if (k > kmax) k = kmax;
  std::vector<double> y(k);
  for (int i = k - 1; i >= 0; --i) {
    double sacc = g[i];
    for (int j = i + 1; j < k; ++j) sacc -= Hc(i, j) * y[j];
    y[i] = sacc / Hc(i, i);
    if (!std::isfinite(y[i]))
      return sps_fail(ctx, SPS_ERR_NONFINITE, "GMRES: non-finite least-squares solution");
  }
  std::memcpy(ctx->h_pinned, y.data(), sizeof(double) * k);
  SPS_CUDA(ctx, cudaMemcpyAsync(d_h1, ctx->h_pinned, sizeof(double) * k, cudaMemcpyHostToDevice,
                                ctx->stream));
  { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
  k_combine<<<gblocks(n), 256, 0, ctx->stream>>>(n, Q, n, k, d_h1, warm ? 1 : 0, x); }
  SPS_LAUNCHED(ctx);
  if (Ax) {
    // A x = A x0 + A V y = (b - beta v_0) + V_{k+1} Hbar y; a zero last norm
    // leaves v_k unwritten and its coefficient zero
    std::vector<double> z(k + 1, 0.0);
    z[0] = -beta;
    for (int j = 0; j < k; ++j)
      for (int i = 0; i <= j + 1; ++i) z[i] += Hbar[(size_t)j * (kmax + 1) + i] * y[j];
    const int cols = (k > 0 && Hbar[(size_t)(k - 1) * (kmax + 1) + k] > 0.0) ? k + 1 : k;
    std::memcpy(ctx->h_pinned + k, z.data(), sizeof(double) * cols);
    SPS_CUDA(ctx, cudaMemcpyAsync(d_h2, ctx->h_pinned + k, sizeof(double) * cols, cudaMemcpyHostToDevice,
                                  ctx->stream));
    SPS_CUDA(ctx, cudaMemcpyAsync(Ax, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
    k_combine<<<gblocks(n), 256, 0, ctx->stream>>>(n, Q, n, cols, d_h2, 1, Ax); }
    SPS_LAUNCHED(ctx);
  }
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *iters = k;
  *relres = res;
  return (res < tol) ? SPS_OK : SPS_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int sps_default_params(sps_params* o) {
  if (!o) return SPS_ERR_INVALID_ARG;
  o->p = 6;
  o->beta = 1.75;
  o->delta = 0.1;
  o->a_c_scale = 1.0;
  o->gmres_tol = 1e-10;
  o->gmres_max = 200;
  o->bbpgd_tol = 1e-8;
  o->bbpgd_max = 10000;
  o->precision = SPS_FP64;
  o->bb_variant = 1;
  o->ir_tol = 0.0;
  o->ir_max = 10;
  o->warm_start = 1;
  o->bb_safeguard = 0;
  o->mobility = SPS_MOB_BIE;
  o->contact_search = SPS_SEARCH_AUTO;
  o->delta_rel = 0.0;
  o->bb_warm = 0;
  o->ir_dw = 1;
  o->lcp_solver = 0;
  return SPS_OK;
}

template <class T>
static int upload(sps_ctx* ctx, T** d, const std::vector<T>& h) {
  SPS_CUDA(ctx, cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(1, h.size())));
  SPS_CUDA(ctx, cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return SPS_OK;
}

extern "C" int sps_create(const sps_params* prm, void* stream, sps_ctx** out) {
  if (!prm || !out) return SPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (prm->p < 1 || prm->p > sps::kMaxP || !(prm->beta > 1.0) || !(prm->gmres_tol > 0) ||
      prm->gmres_max < 1 || !(prm->bbpgd_tol > 0) || prm->bbpgd_max < 1 ||
      (prm->precision != SPS_FP64 && prm->precision != SPS_MIXED && prm->precision != SPS_FP64_DW) ||
      (prm->ir_dw != 0 && prm->ir_dw != 1) ||
      (prm->bb_variant < 1 || prm->bb_variant > 3) || (prm->lcp_solver < 0 || prm->lcp_solver > 2) ||
      !(prm->a_c_scale > 0) ||
      !(prm->delta >= 0) || !(prm->delta_rel >= 0) || !std::isfinite(prm->delta_rel) || prm->ir_tol < 0 || prm->ir_max < 0 ||
      (prm->mobility != SPS_MOB_BIE && prm->mobility != SPS_MOB_IDENTITY) ||
      prm->contact_search < SPS_SEARCH_AUTO || prm->contact_search > SPS_SEARCH_CELLS ||
      (prm->bb_warm < 0 || prm->bb_warm > 2))
    return SPS_ERR_INVALID_ARG;
  sps_ctx* ctx = new sps_ctx();
  ctx->prm = *prm;
  ctx->stream = (cudaStream_t)stream;
  sps::build_tables(prm->p, ctx->T);
  const sps::Tables& T = ctx->T;
  const int P = T.P, NR = T.NR;
  std::vector<double> sS((size_t)3 * P * NR), sK((size_t)3 * P * NR);
  for (int c = 0; c < 3 * P; ++c)
    for (int r = 0; r < NR; ++r) {
      sS[(size_t)c * NR + r] = T.synth[(size_t)c * NR + r] * T.multS[r];
      sK[(size_t)c * NR + r] = T.synth[(size_t)c * NR + r] * T.multK[r];
    }
  auto f32 = [](const std::vector<double>& a) { return std::vector<float>(a.begin(), a.end()); };
  int rc = SPS_OK;
  if ((rc = upload(ctx, &ctx->d_unit_nrm, T.unit_nrm)) || (rc = upload(ctx, &ctx->d_unit_w, T.unit_w)) ||
      (rc = upload(ctx, &ctx->d_anal, T.anal)) || (rc = upload(ctx, &ctx->d_synthS, sS)) ||
      (rc = upload(ctx, &ctx->d_synthK, sK)) || (rc = upload(ctx, &ctx->d_kappa, T.kappa)) || (rc = upload(ctx, &ctx->d_potfac, T.potfac)) ||
      (rc = upload(ctx, &ctx->d_anal32, f32(T.anal))) || (rc = upload(ctx, &ctx->d_synthS32, f32(sS))) ||
      (rc = upload(ctx, &ctx->d_synthK32, f32(sK)))) {
    sps_destroy(ctx);
    return rc;
  }
  {
    // transposed self matrices (adjoint): analysis^T (3P x NR), synthesis^T (NR x 3P)
    std::vector<double> aT((size_t)3 * P * NR), sST((size_t)NR * 3 * P), sKT((size_t)NR * 3 * P);
    for (int r = 0; r < NR; ++r)
      for (int c = 0; c < 3 * P; ++c) {
        aT[(size_t)c * NR + r] = T.anal[(size_t)r * 3 * P + c];
        sST[(size_t)r * 3 * P + c] = sS[(size_t)c * NR + r];
        sKT[(size_t)r * 3 * P + c] = sK[(size_t)c * NR + r];
      }
    if ((rc = upload(ctx, &ctx->d_analT, aT)) || (rc = upload(ctx, &ctx->d_synthST, sST)) ||
        (rc = upload(ctx, &ctx->d_synthKT, sKT)) || (rc = sps_build_field_maps(ctx)) ||
        (rc = sps_sht_tc_upload(ctx, ctx->tcA, T.anal, NR, 3 * P)) ||
        (rc = sps_sht_tc_upload(ctx, ctx->tcS, sS, 3 * P, NR)) ||
        (rc = sps_sht_tc_upload(ctx, ctx->tcK, sK, 3 * P, NR))) {
      sps_destroy(ctx);
      return rc;
    }
  }
  {
    size_t c = 0;
    if ((rc = sps_grow(ctx, &ctx->d_sc, c, (size_t)2 * kRedBlocks + 8))) {
      sps_destroy(ctx);
      return rc;
    }
  }
  if (cudaMallocHost((void**)&ctx->h_pinned, sizeof(double) * 4096) != cudaSuccess) {
    cudaGetLastError();
    sps_destroy(ctx);
    return SPS_ERR_CUDA;
  }
  *out = ctx;
  return SPS_OK;
}

extern "C" int sps_destroy(sps_ctx* ctx) {
  if (!ctx) return SPS_OK;
  void* bufs[] = {ctx->d_unit_nrm, ctx->d_unit_w, ctx->d_anal, ctx->d_synthS, ctx->d_synthK,
                  ctx->d_kappa, ctx->d_potfac, ctx->d_anal32, ctx->d_synthS32, ctx->d_synthK32, ctx->d_pos, ctx->d_rad,
                  ctx->d_X, ctx->d_Nrm, ctx->d_W, ctx->d_rel32, ctx->d_N32, ctx->d_W32, ctx->d_chi, ctx->d_clo,
                  ctx->d_near_ptr, ctx->d_near_idx, ctx->d_close_node, ctx->d_close_ptr,
                  ctx->d_close_src, ctx->d_coef, ctx->d_fcoef, ctx->d_mom,
                  ctx->d_tmp3, ctx->d_sig32, ctx->d_part, ctx->d_Q, ctx->d_w, ctx->d_h, ctx->d_red,
                  ctx->d_rho, ctx->d_zeta, ctx->d_zeta_nc, ctx->d_b, ctx->d_u, ctx->d_r, ctx->d_dz, ctx->d_cij,
                  ctx->d_cphi, ctx->d_cn, ctx->d_ccount, ctx->d_cptr, ctx->d_inc_ptr, ctx->d_inc,
                  ctx->d_cub, ctx->d_keys, ctx->d_vals, ctx->d_keys2, ctx->d_vals2, ctx->d_gam,
                  ctx->d_g, ctx->d_gam_new, ctx->d_g_new, ctx->d_q, ctx->d_Mg, ctx->d_FT,
                  ctx->d_Unc, ctx->d_Uc};
  for (void* b : bufs)
    if (b) cudaFree(b);
  void* more[] = {ctx->d_analT, ctx->d_synthST, ctx->d_synthKT, ctx->d_coefbar, ctx->d_ebar,
                  ctx->d_sigtot, ctx->d_ubar, ctx->d_sbar, ctx->d_lam, ctx->d_rbar,
                  ctx->d_ccount2, ctx->d_inc_cnt, ctx->d_cl_key, ctx->d_cl_id, ctx->d_cl_key2,
                  ctx->d_cl_id2, ctx->d_cl_range, ctx->d_cl_f, ctx->d_cl_d, ctx->d_cl_part,
                  ctx->d_flag, ctx->d_bbpart, ctx->d_F3, ctx->d_iFT, ctx->d_sc, ctx->tcA.d,
                  ctx->tcS.d, ctx->tcK.d, ctx->d_tcflag, ctx->d_order,
                  ctx->d_adj6a, ctx->d_adj6b, ctx->d_adjc, ctx->d_gam_best, ctx->d_aux_best,
                  ctx->d_Pb, ctx->d_Px, ctx->d_fcoef32, ctx->d_fcoefdw, ctx->d_prev_ij, ctx->d_prev_gam,
                  ctx->d_dwsrc, ctx->d_rot, ctx->d_sigloc, ctx->d_tcsplit, ctx->d_near_rev,
                  ctx->d_near_geo, ctx->d_near_buf, ctx->d_wcount, ctx->d_wptr, ctx->d_inc_fill,
                  ctx->d_cl_fill, ctx->d_scan_tot, ctx->d_apgd};
  for (void* b : more)
    if (b) cudaFree(b);
  for (sps_ctx::Sparse* m : {&ctx->fmK, &ctx->fmS, &ctx->fmKt, &ctx->fmSt}) {
    cudaFree(m->rp);
    cudaFree(m->ci);
    cudaFree(m->v);
  }
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
  return SPS_OK;
}

extern "C" const char* sps_last_error(const sps_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

static int check_finite_host(sps_ctx* ctx, const double* d, long long n, const char* what) {
  std::vector<double> h(n);
  SPS_CUDA(ctx, cudaMemcpyAsync(h.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(h[i])) return sps_fail(ctx, SPS_ERR_NONFINITE, std::string(what) + " is not finite");
  return SPS_OK;
}

extern "C" int sps_set_orientation(sps_ctx* ctx, int n, const double* Q) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  ctx->have_geom = false;          // nodes and normals depend on the orientation
  ctx->zeta_n = ctx->zeta_nc_n = 0;
  ctx->prev_nc = 0;
  if (!Q) {
    ctx->rot_n = 0;
    return SPS_OK;
  }
  if (n < 1) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "set_orientation: n must be positive");
  std::vector<double> h(9 * (size_t)n);
  SPS_CUDA(ctx, cudaMemcpyAsync(h.data(), Q, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < n; ++i) {
    const double* q = h.data() + 9 * (size_t)i;
    for (int k = 0; k < 9; ++k)
      if (!std::isfinite(q[k])) return sps_fail(ctx, SPS_ERR_NONFINITE, "orientation not finite");
    // Q^T Q = I and det Q = +1, to 1e-12
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double d = 0.0;
        for (int r = 0; r < 3; ++r) d += q[3 * r + a] * q[3 * r + b];
        if (std::fabs(d - (a == b ? 1.0 : 0.0)) > 1e-12)
          return sps_fail(ctx, SPS_ERR_INVALID_ARG, "orientation is not orthogonal");
      }
    const double det = q[0] * (q[4] * q[8] - q[5] * q[7]) - q[1] * (q[3] * q[8] - q[5] * q[6]) +
                       q[2] * (q[3] * q[7] - q[4] * q[6]);
    if (!(det > 0)) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "orientation is a reflection");
  }
  SPS_TRY(sps_grow(ctx, &ctx->d_rot, ctx->cap_rot, 9 * (size_t)n));
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_rot, Q, sizeof(double) * 9 * n, cudaMemcpyDeviceToDevice, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->rot_n = n;
  return SPS_OK;
}

extern "C" int sps_set_walls(sps_ctx* ctx, int n_walls, const double* walls) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (n_walls < 0 || n_walls > kMaxWalls || (n_walls > 0 && !walls))
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "set_walls: 0 to 8 walls");
  SpsWalls W;
  W.n = n_walls;
  for (int w = 0; w < n_walls; ++w) {
    const double* r = walls + 4 * w;
    for (int k = 0; k < 4; ++k)
      if (!std::isfinite(r[k])) return sps_fail(ctx, SPS_ERR_NONFINITE, "set_walls: not finite");
    const double nn = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    if (std::fabs(nn - 1.0) > 1e-12) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "set_walls: normal not unit");
    for (int k = 0; k < 4; ++k) W.w[w][k] = r[k];
  }
  ctx->walls = W;
  ctx->prev_nc = 0;     // the previous list's wall rows refer to the old walls
  return SPS_OK;
}

// oriented grids are not differentiated (the adjoint kernels use lab-frame
// VSH maps)
static int no_orientation(sps_ctx* ctx, const char* what) {
  if (ctx->rot_n > 0)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, std::string(what) + ": not available with grid orientations");
  return SPS_OK;
}

extern "C" int sps_set_geometry(sps_ctx* ctx, int n, const double* pos, const double* radii) {
  if (!ctx || n < 1 || !pos || !radii) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "set_geometry: bad argument");
  if (ctx->rot_n > 0 && ctx->rot_n != n)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "set_geometry: the grid orientation is set for another sphere count");
  const int P = ctx->T.P;
  const long long NP = (long long)n * P;
  {
    std::vector<double> h(4 * (size_t)n);
    SPS_CUDA(ctx, cudaMemcpyAsync(h.data(), pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA(ctx, cudaMemcpyAsync(h.data() + 3 * n, radii, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < h.size(); ++i)
      if (!std::isfinite(h[i])) return sps_fail(ctx, SPS_ERR_NONFINITE, "positions or radii not finite");
    for (int i = 0; i < n; ++i)
      if (!(h[3 * n + i] > 0)) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "radii must be positive");
  }
  if (n > ctx->capN) {
    double** d64[] = {&ctx->d_pos, &ctx->d_rad, &ctx->d_X, &ctx->d_Nrm, &ctx->d_W, &ctx->d_coef,
                      &ctx->d_fcoef, &ctx->d_mom, &ctx->d_tmp3, &ctx->d_rho, &ctx->d_zeta,
                      &ctx->d_zeta_nc, &ctx->d_b,
                      &ctx->d_u, &ctx->d_r, &ctx->d_dz, &ctx->d_FT, &ctx->d_Unc, &ctx->d_Uc,
                      &ctx->d_coefbar, &ctx->d_ebar, &ctx->d_sigtot, &ctx->d_ubar, &ctx->d_sbar,
                      &ctx->d_lam, &ctx->d_rbar};
    for (auto p : d64) {
      cudaFree(*p);
      *p = nullptr;
    }
    float** d32[] = {&ctx->d_rel32, &ctx->d_N32, &ctx->d_W32, &ctx->d_sig32, &ctx->d_chi, &ctx->d_clo,
                     &ctx->d_fcoef32};
    cudaFree(ctx->d_fcoefdw);
    ctx->d_fcoefdw = nullptr;
    for (auto p : d32) {
      cudaFree(*p);
      *p = nullptr;
    }
    cudaFree(ctx->d_near_ptr);
    ctx->d_near_ptr = nullptr;
    size_t c;
    const size_t E = ctx->T.E, NR = ctx->T.NR;
    struct {
      double** p;
      size_t n;
    } a64[] = {{&ctx->d_pos, 3 * (size_t)n}, {&ctx->d_rad, (size_t)n}, {&ctx->d_X, 3 * (size_t)NP},
               {&ctx->d_Nrm, 3 * (size_t)NP}, {&ctx->d_W, (size_t)NP}, {&ctx->d_coef, (size_t)n * NR},
               {&ctx->d_fcoef, (size_t)n * E * sps::kFieldsK * 2}, {&ctx->d_mom, 6 * (size_t)n},
               {&ctx->d_tmp3, 3 * (size_t)NP}, {&ctx->d_rho, 3 * (size_t)NP},
               {&ctx->d_zeta, 3 * (size_t)NP}, {&ctx->d_zeta_nc, 3 * (size_t)NP},
               {&ctx->d_b, 3 * (size_t)NP}, {&ctx->d_u, 3 * (size_t)NP},
               {&ctx->d_r, 3 * (size_t)NP}, {&ctx->d_dz, 3 * (size_t)NP}, {&ctx->d_FT, 6 * (size_t)n},
               {&ctx->d_Unc, 6 * (size_t)n}, {&ctx->d_Uc, 6 * (size_t)n},
               {&ctx->d_coefbar, (size_t)n * NR}, {&ctx->d_ebar, (size_t)n * E * sps::kFieldsK * 2},
               {&ctx->d_sigtot, 3 * (size_t)NP}, {&ctx->d_ubar, 3 * (size_t)NP}, {&ctx->d_sbar, 3 * (size_t)NP},
               {&ctx->d_lam, 3 * (size_t)NP}, {&ctx->d_rbar, 3 * (size_t)NP}};
    for (auto& e : a64) {
      c = 0;
      SPS_TRY(sps_grow(ctx, e.p, c, e.n));
    }
    struct {
      float** p;
      size_t n;
    } a32[] = {{&ctx->d_rel32, 3 * (size_t)NP}, {&ctx->d_N32, 3 * (size_t)NP}, {&ctx->d_W32, (size_t)NP},
               {&ctx->d_sig32, 3 * (size_t)NP}, {&ctx->d_chi, 3 * (size_t)n}, {&ctx->d_clo, 3 * (size_t)n},
               {&ctx->d_fcoef32, (size_t)n * E * sps::kFieldsK * 2}};
    for (auto& e : a32) {
      c = 0;
      SPS_TRY(sps_grow(ctx, e.p, c, e.n));
    }
    c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_fcoefdw, c, (size_t)n * E * sps::kFieldsK * 2));
    c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_near_ptr, c, (size_t)n + 1));
    ctx->capN = n;
  }
  if (n != ctx->N) ctx->zeta_nc_n = 0;
  ctx->N = n;
  ctx->NP = (int)NP;
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_pos, pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, ctx->stream));
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_rad, radii, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  SPS_TRY(sps_launch_grid(ctx));
  SPS_TRY(sps_launch_near_lists(ctx));
  SPS_TRY(sps_launch_close_lists(ctx));
  SPS_TRY(sps_launch_near_rev(ctx));
  ctx->have_geom = true;
  return SPS_OK;
}

extern "C" int sps_nodes(sps_ctx* ctx, double* X, double* normals, double* weights, int* np_out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!ctx->have_geom) return sps_fail(ctx, SPS_ERR_NO_GEOMETRY, "no geometry");
  const size_t NP = ctx->NP;
  if (X) SPS_CUDA(ctx, cudaMemcpyAsync(X, ctx->d_X, 3 * NP * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  if (normals)
    SPS_CUDA(ctx, cudaMemcpyAsync(normals, ctx->d_Nrm, 3 * NP * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  if (weights) SPS_CUDA(ctx, cudaMemcpyAsync(weights, ctx->d_W, NP * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  if (np_out) *np_out = (int)NP;
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

extern "C" int sps_geometry_counts(const sps_ctx* ctx, int* n_near_pairs, int* n_close_entries) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!ctx->have_geom) return SPS_ERR_NO_GEOMETRY;
  if (n_near_pairs) *n_near_pairs = ctx->n_near;
  if (n_close_entries) *n_close_entries = ctx->n_close_src;
  return SPS_OK;
}

extern "C" int sps_near_lists(sps_ctx* ctx, int* near_ptr, int* near_idx) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!ctx->have_geom) return sps_fail(ctx, SPS_ERR_NO_GEOMETRY, "no geometry");
  if (near_ptr)
    SPS_CUDA(ctx, cudaMemcpyAsync(near_ptr, ctx->d_near_ptr, sizeof(int) * (ctx->N + 1),
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  if (near_idx && ctx->n_near > 0)
    SPS_CUDA(ctx, cudaMemcpyAsync(near_idx, ctx->d_near_idx, sizeof(int) * ctx->n_near,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

extern "C" int sps_layer_apply(sps_ctx* ctx, int op, const double* sigma, double* out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!ctx->have_geom) return sps_fail(ctx, SPS_ERR_NO_GEOMETRY, "no geometry");
  if (op < SPS_OP_S || op > SPS_OP_A || !sigma || !out)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "layer_apply: bad argument");
  SPS_TRY(sps_layer(ctx, op, sigma, out, ctx->prm.precision == SPS_MIXED));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return sps_sht_tc_status(ctx);
}

// ---------------------------------------------------------------------------
// mobility solve on the current geometry
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Initial guesses from earlier solves with the same operator (one geometry,
// inside one collision step): an orthonormal basis Pb of the products A x of
// earlier solutions and the matching combinations Px of those solutions
// (A Px_k = Pb_k to rounding; GMRES returns A x from its Arnoldi relation).
// For a new b the guess x0 = Px (Pb^T b) has the residual b - Pb Pb^T b, the
// smallest over combinations of the earlier solutions, known without an
// application of A.  Every solve still runs GMRES to gmres_tol; only its
// starting point changes.
// ---------------------------------------------------------------------------
constexpr int kProjMax = 16;

static int proj_ensure(sps_ctx* ctx, long long n) {
  if (ctx->proj_n == n && ctx->d_Pb) return SPS_OK;
  cudaFree(ctx->d_Pb);
  cudaFree(ctx->d_Px);
  ctx->d_Pb = ctx->d_Px = nullptr;
  size_t c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_Pb, c, (size_t)kProjMax * n));
  c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_Px, c, (size_t)kProjMax * n));
  ctx->proj_n = n;
  ctx->proj_m = 0;
  return SPS_OK;
}

// x = Px Pb^T b and r = b - Pb Pb^T b (= b - A x)
static int proj_guess(sps_ctx* ctx, const double* b, double* x, double* r, bool* used) {
  *used = false;
  const int m = ctx->proj_m;
  const long long n = 3LL * ctx->NP;
  if (!ctx->proj_on || m == 0 || ctx->proj_n != n) return SPS_OK;
  SPS_TRY(ensure_gmres(ctx, n, ctx->prm.gmres_max));
  SPS_TRY(multidot_dev(ctx, ctx->d_Pb, n, m, b, n, ctx->d_h, ctx->d_red));
  SPS_CUDA(ctx, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
  k_combine<<<gblocks(n), 256, 0, ctx->stream>>>(n, ctx->d_Px, n, m, ctx->d_h, 0, x);
  k_sub_proj<<<gblocks(n), 256, 0, ctx->stream>>>(n, ctx->d_Pb, n, m, ctx->d_h, r); }
  ctx->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sps_fail(ctx, SPS_ERR_CUDA, cudaGetErrorString(e));
  *used = true;
  return SPS_OK;
}

// adds the pair (b, x) with b = A x
static int proj_add(sps_ctx* ctx, const double* b, const double* x) {
  if (!ctx->proj_on) return SPS_OK;
  const long long n = 3LL * ctx->NP;
  SPS_TRY(proj_ensure(ctx, n));
  SPS_TRY(ensure_gmres(ctx, n, ctx->prm.gmres_max));
  int m = ctx->proj_m;
  int slot = m;
  if (m == kProjMax) {
    // full: the oldest pair gives way (the remaining columns stay orthonormal)
    slot = ctx->proj_old;
    ctx->proj_old = (ctx->proj_old + 1) % kProjMax;
    SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_Pb + (size_t)slot * n, 0, sizeof(double) * n, ctx->stream));
    SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_Px + (size_t)slot * n, 0, sizeof(double) * n, ctx->stream));
  }
  double* pb = ctx->d_Pb + (size_t)slot * n;
  double* px = ctx->d_Px + (size_t)slot * n;
  double bb = 0.0;
  SPS_TRY(sps_dot(ctx, b, b, n, &bb));
  if (!(bb > 0.0) || !std::isfinite(bb)) return SPS_OK;
  SPS_CUDA(ctx, cudaMemcpyAsync(pb, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  SPS_CUDA(ctx, cudaMemcpyAsync(px, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  // classical Gram-Schmidt, twice, against every stored column (a zeroed
  // slot being refilled contributes nothing)
  for (int pass = 0; pass < 2 && m > 0; ++pass) {
    if (slot < m) {
      // the slot's own (new) content must not be projected out of itself
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_dz, pb, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
      SPS_CUDA(ctx, cudaMemsetAsync(pb, 0, sizeof(double) * n, ctx->stream));
      SPS_TRY(multidot_dev(ctx, ctx->d_Pb, n, m, ctx->d_dz, n, ctx->d_h, ctx->d_red));
      SPS_CUDA(ctx, cudaMemcpyAsync(pb, ctx->d_dz, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_dz, px, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
      SPS_CUDA(ctx, cudaMemsetAsync(px, 0, sizeof(double) * n, ctx->stream));
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_sub_proj<<<gblocks(n), 256, 0, ctx->stream>>>(n, ctx->d_Pb, n, m, ctx->d_h, pb);
      k_sub_proj<<<gblocks(n), 256, 0, ctx->stream>>>(n, ctx->d_Px, n, m, ctx->d_h, ctx->d_dz); }
      ctx->launches += 2;
      SPS_CUDA(ctx, cudaMemcpyAsync(px, ctx->d_dz, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
      continue;
    }
    SPS_TRY(multidot_dev(ctx, ctx->d_Pb, n, m, pb, n, ctx->d_h, ctx->d_red));
    { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
    k_sub_proj<<<gblocks(n), 256, 0, ctx->stream>>>(n, ctx->d_Pb, n, m, ctx->d_h, pb);
    k_sub_proj<<<gblocks(n), 256, 0, ctx->stream>>>(n, ctx->d_Px, n, m, ctx->d_h, px); }
    ctx->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sps_fail(ctx, SPS_ERR_CUDA, cudaGetErrorString(e));
  }
  double nn = 0.0;
  SPS_TRY(sps_dot(ctx, pb, pb, n, &nn));
  // b (nearly) in the span already: normalising what is left would amplify
  // the rounding of A Px = Pb
  if (!(nn > 1e-12 * bb) || !std::isfinite(nn)) return SPS_OK;
  const double inv = 1.0 / std::sqrt(nn);
  { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
  k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, inv, pb, 0.0, nullptr, pb);
  k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, inv, px, 0.0, nullptr, px); }
  ctx->launches += 2;
  if (slot == m) ctx->proj_m = m + 1;
  return SPS_OK;
}

// the projection space lives for one collision step
// SPS_PROJ_KEEP = 1 keeps the basis from one step to the next (same node
// count); measured on 1,000 spheres it raised GMRES iterations per step from
// 150 to 182 (the previous step's pairs are worse starting points than the
// current step's), so each step starts an empty basis.
#ifndef SPS_PROJ_KEEP
#define SPS_PROJ_KEEP 0
#endif
struct ProjScope {
  sps_ctx* c;
  explicit ProjScope(sps_ctx* ctx) : c(ctx) {
    c->proj_on = ctx->prm.warm_start != 0;
    if (!SPS_PROJ_KEEP || !c->proj_on || c->proj_n != 3LL * ctx->NP) {
      c->proj_m = 0;
      c->proj_old = 0;
    }
  }
  ~ProjScope() { c->proj_on = false; }
};

// zeta: receives mu = rho + zeta, where zeta is the density unknown of eq.
// rigidbodyrho; with warm it holds an initial guess on entry (a previous
// solution for similar forces).  mu solves (I/2 + K + L)[mu] = L[rho]: since
// (I/2 + K + L)[rho] - (I/2 + K)[rho] = L[rho] this is eq. rigidbodyrho's
// discrete solve, with a right-hand side that needs only the sphere moments
// of rho instead of a traction application.  The density of eq. velS is mu.
static int mobility_solve(sps_ctx* ctx, const double* FT, double* UO, sps_stats* st, double* zeta,
                          bool warm) {
  const long long n = 3LL * ctx->NP;
  const bool mixed = ctx->prm.precision == SPS_MIXED;
  const bool refine = mixed && ctx->prm.ir_tol > 0;
  SPS_TRY(sps_launch_rho(ctx, FT, ctx->d_rho));
  // b = L[rho]: the unknown is mu = rho + zeta, (I/2 + K + L)[mu] = L[rho]
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_b, 0, sizeof(double) * n, ctx->stream));
  SPS_TRY(sps_launch_moments(ctx, ctx->d_rho, ctx->d_mom));
  SPS_TRY(sps_launch_add_L(ctx, ctx->d_mom, ctx->d_b));
  int its = 0;
  double res = 0.0;
  bool projected = false;
  // with refinement the stored pairs would not match the refined solutions:
  // the projection then stays off
  if (!refine) SPS_TRY(proj_guess(ctx, ctx->d_b, zeta, ctx->d_r, &projected));
  // A zeta lands in d_u (free until the velocity is formed)
  int rc = gmres(ctx, ctx->d_b, zeta, warm || projected, ctx->prm.gmres_tol, ctx->prm.gmres_max, mixed,
                 &its, &res, projected ? ctx->d_r : nullptr, (refine || !ctx->proj_on) ? nullptr : ctx->d_u);
  if (rc != SPS_OK && rc != SPS_ERR_NOT_CONVERGED) return rc;
  int total_its = its;
  double final_res = res;
  if (refine) {
    // iterative refinement against the FP64 operator: r = b - A zeta
    double bb = 0.0;
    SPS_TRY(sps_dot(ctx, ctx->d_b, ctx->d_b, n, &bb));
    const double nb = std::sqrt(bb);
    int sweep = 0;
    for (; sweep < ctx->prm.ir_max; ++sweep) {
      SPS_TRY(apply_A(ctx, zeta, ctx->d_r, false));
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, 1.0, ctx->d_b, -1.0, ctx->d_r, ctx->d_r); }
      SPS_LAUNCHED(ctx);
      double rr = 0.0;
      SPS_TRY(sps_dot(ctx, ctx->d_r, ctx->d_r, n, &rr));
      final_res = nb > 0 ? std::sqrt(rr) / nb : 0.0;
      if (final_res < ctx->prm.ir_tol) break;
      // the correction need only shrink the residual by the factor still
      // missing (with a margin), never below gmres_tol: one sweep's reduction
      // is limited by the FP32 operator's own error anyway
      const double need = ctx->prm.ir_tol / std::max(final_res, 1e-300);
      const double ctol = std::min(1e-1, std::max(ctx->prm.gmres_tol, 0.5 * need));
      int its2 = 0;
      double res2 = 0;
      int rc2 = gmres(ctx, ctx->d_r, ctx->d_dz, false, ctol, ctx->prm.gmres_max, true, &its2, &res2);
      if (rc2 != SPS_OK && rc2 != SPS_ERR_NOT_CONVERGED) return rc2;
      total_its += its2;
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_axpby<<<gblocks(n), 256, 0, ctx->stream>>>(n, 1.0, zeta, 1.0, ctx->d_dz, zeta); }
      SPS_LAUNCHED(ctx);
    }
    if (st) st->ir_sweeps += sweep;
    rc = (final_res < ctx->prm.ir_tol) ? SPS_OK : SPS_ERR_NOT_CONVERGED;
  }
  if (!refine && rc == SPS_OK) SPS_TRY(proj_add(ctx, ctx->d_u, zeta));
  // u = S[rho + zeta] = S[mu]
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_tmp3, zeta, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  SPS_TRY(sps_layer(ctx, SPS_OP_S, ctx->d_tmp3, ctx->d_u, mixed && !refine));
  SPS_TRY(sps_launch_moments(ctx, ctx->d_u, ctx->d_mom));
  SPS_TRY(sps_launch_extract(ctx, ctx->d_mom, UO));
  if (mixed) SPS_TRY(sps_sht_tc_status(ctx));
  if (st) {
    st->mobility_solves += 1;
    st->gmres_iters += total_its;
    st->gmres_iters_max = std::max(st->gmres_iters_max, total_its);
    st->gmres_res_max = std::max(st->gmres_res_max, final_res);
  }
  return rc;
}

static void stats_begin(sps_ctx* ctx, sps_stats* st, long long* l0) {
  if (st) std::memset(st, 0, sizeof(*st));
  *l0 = ctx->launches;
  ctx->stats_layer0 = ctx->layer_applies;
}
static int stats_end(sps_ctx* ctx, sps_stats* st, long long l0, int rc) {
  if (st) {
    st->status = rc;
    st->kernel_launches = ctx->launches - l0;
    st->layer_applies = (int)(ctx->layer_applies - ctx->stats_layer0);
    st->n_near_pairs = ctx->n_near;
  }
  return rc;
}

extern "C" int sps_mobility_apply(sps_ctx* ctx, int n, const double* pos, const double* radii,
                                  const double* FT, double* UO, sps_stats* st) {
  if (!ctx || !FT || !UO || n < 1 || !pos || !radii)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "mobility_apply: bad argument");
  long long l0;
  stats_begin(ctx, st, &l0);
  if (ctx->prm.mobility == SPS_MOB_IDENTITY) {
    int rc = sps_check_inputs(ctx, n, pos, radii, FT);
    if (rc == SPS_OK) rc = sps_launch_identity_U(ctx, n, FT, nullptr, UO);
    if (rc == SPS_OK) {
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) rc = sps_fail(ctx, SPS_ERR_CUDA, cudaGetErrorString(e));
    }
    return stats_end(ctx, st, l0, rc);
  }
  int rc = sps_set_geometry(ctx, n, pos, radii);
  if (rc == SPS_OK) rc = check_finite_host(ctx, FT, 6LL * n, "force/torque");
  // warm start from the previous solve on a suspension of the same size
  const bool warm = ctx->prm.warm_start && ctx->zeta_n == ctx->NP;
  if (rc == SPS_OK) rc = mobility_solve(ctx, FT, UO, st, ctx->d_zeta, warm);
  ctx->zeta_n = (rc == SPS_OK) ? ctx->NP : 0;
  if (rc == SPS_OK || rc == SPS_ERR_NOT_CONVERGED) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = sps_fail(ctx, SPS_ERR_CUDA, cudaGetErrorString(e));
  }
  return stats_end(ctx, st, l0, rc);
}

extern "C" int sps_build_contacts(sps_ctx* ctx, int n, const double* pos, const double* radii,
                                  int* n_contacts) {
  if (!ctx || n < 1 || !pos || !radii) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "build_contacts: bad argument");
  SPS_TRY(sps_launch_contacts(ctx, n, pos, radii));
  ctx->c_N = n;
  if (n_contacts) *n_contacts = ctx->n_c;
  return SPS_OK;
}

extern "C" int sps_get_contacts(sps_ctx* ctx, int* ij, double* phi, double* normals) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  const size_t nc = ctx->n_c;
  if (nc == 0) return SPS_OK;
  if (ij) SPS_CUDA(ctx, cudaMemcpyAsync(ij, ctx->d_cij, nc * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  if (phi) SPS_CUDA(ctx, cudaMemcpyAsync(phi, ctx->d_cphi, nc * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  if (normals)
    SPS_CUDA(ctx, cudaMemcpyAsync(normals, ctx->d_cn, nc * 24, cudaMemcpyDeviceToDevice, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

extern "C" int sps_contact_force(sps_ctx* ctx, const double* gamma, double* FT) {
  if (!ctx || !FT || (ctx->n_c && !gamma)) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "contact_force");
  if (ctx->c_N == 0) return sps_fail(ctx, SPS_ERR_NO_GEOMETRY, "no contact list");
  SPS_TRY(sps_launch_D(ctx, gamma, FT));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

extern "C" int sps_contact_rate(sps_ctx* ctx, const double* UO, double* out) {
  if (!ctx || !UO || (ctx->n_c && !out)) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "contact_rate");
  SPS_TRY(sps_launch_DT(ctx, UO, out));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

// ---------------------------------------------------------------------------
// collision-resolved step
// ---------------------------------------------------------------------------
static int ensure_bb(sps_ctx* ctx, int nc) {
  if (nc <= ctx->cap_bb && ctx->d_gam) return SPS_OK;
  double** v[] = {&ctx->d_gam, &ctx->d_g, &ctx->d_gam_new, &ctx->d_g_new, &ctx->d_q, &ctx->d_Mg};
  for (auto p : v) {
    cudaFree(*p);
    *p = nullptr;
    size_t c = 0;
    SPS_TRY(sps_grow(ctx, p, c, (size_t)std::max(nc, 1)));
  }
  ctx->cap_bb = std::max(nc, 1);
  return SPS_OK;
}

// out = M gamma = D^T M D gamma; leaves M D gamma in d_Uc.  warm: start GMRES
// from the density of the previous M gamma solve (same contact geometry).
static int apply_M(sps_ctx* ctx, const double* gam, double* out, sps_stats* st, bool warm) {
  SPS_TRY(sps_launch_D(ctx, gam, ctx->d_FT));
  int rc = mobility_solve(ctx, ctx->d_FT, ctx->d_Uc, st, ctx->d_zeta, warm);
  ctx->zeta_n = 0;   // d_zeta now holds a contact-force solve
  if (rc != SPS_OK && rc != SPS_ERR_NOT_CONVERGED) return rc;
  SPS_TRY(sps_launch_DT(ctx, ctx->d_Uc, out));
  return rc;
}

static int read5(sps_ctx* ctx, double out[5]) {
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, sps_bb_out(ctx), 5 * sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::memcpy(out, ctx->h_pinned, 5 * sizeof(double));
  for (int i = 0; i < 5; ++i)
    if (!std::isfinite(out[i])) return sps_fail(ctx, SPS_ERR_NONFINITE, "BBPGD: non-finite residual");
  return SPS_OK;
}

static int bb_stats(sps_ctx* ctx, const double* gn, const double* ggn, const double* go,
                    const double* ggo, double out[5]) {
  SPS_TRY(sps_bb_stats_dev(ctx, gn, ggn, go, ggo));
  return read5(ctx, out);
}

struct BBResult {
  int iters = 0;
  int best_iter = 0;    // iterate returned (differs from iters after a failure)
  double phi = 0.0;
  int bb_rc = SPS_OK;   // BREAKDOWN / NOT_CONVERGED of Algorithm 1 itself
  int worst = SPS_OK;   // NOT_CONVERGED of an inner mobility solve
};

// Algorithm 1 from gamma_0 = 0 on the current contact list, q in d_q.
//   mul_g():             d_Mg = M d_g   (for alpha_0 = g^T g / g^T M g)
//   step(alpha, j, s5):  d_gam_new = max(d_gam - alpha d_g, 0),
//                        d_g_new = M d_gam_new + q, s5 = the five statistics
// Each returns an sps_status; NOT_CONVERGED (an inner solve) is recorded and
// the iteration goes on.  Returns the first hard error, else SPS_OK with the
// outcome in r; d_gam / d_g hold the last iterate.
template <class MulG, class Step, class MulGam>
static int bbpgd_run(sps_ctx* ctx, int nc, sps_stats* st, MulG mul_g, Step step, BBResult& r,
                     double* aux, size_t aux_len, bool warm0, MulGam mul_gam) {
  int rc = SPS_OK;
  if (warm0) {
    // gamma_0 (in d_gam) from the caller: g_0 = M gamma_0 + q
    rc = mul_gam();
    if (rc != SPS_OK && rc != SPS_ERR_NOT_CONVERGED) return rc;
    if (rc) r.worst = rc;
    if (st) st->mvops += 1;
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_add<<<(nc + 255) / 256, 256, 0, ctx->stream>>>(nc, ctx->d_Mg, ctx->d_q, ctx->d_g); }
    SPS_LAUNCHED(ctx);
  } else {
    SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_gam, 0, sizeof(double) * nc, ctx->stream));
    SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_g, ctx->d_q, sizeof(double) * nc, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  }
  double s5[5];
  SPS_TRY(bb_stats(ctx, ctx->d_gam, ctx->d_g, nullptr, nullptr, s5));
  if (warm0) {
    // keep the initial guess only if its min-map residual beats gamma_0 = 0's
    // (a guess from a step that resolved large overlaps can be far worse)
    double z5[5];
    SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_gam_new, 0, sizeof(double) * nc, ctx->stream));
    SPS_TRY(bb_stats(ctx, ctx->d_gam_new, ctx->d_q, nullptr, nullptr, z5));
    if (!(s5[0] < z5[0])) {
      warm0 = false;
      SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_gam, 0, sizeof(double) * nc, ctx->stream));
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_g, ctx->d_q, sizeof(double) * nc, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
      if (aux) SPS_CUDA(ctx, cudaMemsetAsync(aux, 0, sizeof(double) * aux_len, ctx->stream));
      std::memcpy(s5, z5, sizeof(s5));
    }
  }
  r.phi = std::sqrt(s5[0]);
  const double tol = ctx->prm.bbpgd_tol;
  if (r.phi < tol) return SPS_OK;
  if (aux) {
    SPS_TRY(sps_grow(ctx, &ctx->d_gam_best, ctx->cap_gam_best, (size_t)std::max(nc, 1)));
    SPS_TRY(sps_grow(ctx, &ctx->d_aux_best, ctx->cap_aux_best, std::max<size_t>(aux_len, 1)));
    if (warm0) {   // the start is the first candidate for the best iterate
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_gam_best, ctx->d_gam, sizeof(double) * nc,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_aux_best, aux, sizeof(double) * aux_len,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
  double alpha = 0.0;
  if (warm0 && ctx->prm.bb_warm == 2 && ctx->prev_alpha > 0) {
    alpha = ctx->prev_alpha;   // the previous step's last step length: no product M g_0
  } else {
    rc = mul_g();
    if (rc != SPS_OK && rc != SPS_ERR_NOT_CONVERGED) return rc;
    if (rc) r.worst = rc;
    if (st) st->mvops += 1;
    double gMg = 0.0;
    SPS_TRY(sps_dot(ctx, ctx->d_g, ctx->d_Mg, nc, &gMg));
    if (!(gMg > 0)) {
      r.bb_rc = SPS_ERR_BREAKDOWN;
      return SPS_OK;
    }
    alpha = s5[4] / gMg;
  }
  ctx->bb_alpha_last = alpha;
  // divergence: an indefinite discrete M (nearly touching spheres at low
  // order) makes the projected steps grow without bound
  const double phi_limit = 1e6 * std::max(r.phi, tol);
  // with aux (the vector holding M D gamma of the current iterate), the
  // iterate of smallest residual is kept and returned if the loop fails
  double best_phi = r.phi;
  int best_j = 0;
  auto fail = [&](int code, int j) -> int {
    r.bb_rc = code;
    if (aux && best_j != j) {
      if (best_j == 0 && !warm0) {
        SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_gam, 0, sizeof(double) * nc, ctx->stream));
        SPS_CUDA(ctx, cudaMemsetAsync(aux, 0, sizeof(double) * aux_len, ctx->stream));
      } else {
        SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_gam, ctx->d_gam_best, sizeof(double) * nc,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
        SPS_CUDA(ctx, cudaMemcpyAsync(aux, ctx->d_aux_best, sizeof(double) * aux_len,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
      }
      r.phi = best_phi;
      r.best_iter = best_j;
    }
    return SPS_OK;
  };
  int j = 1;
  for (; j <= ctx->prm.bbpgd_max; ++j) {
    rc = step(alpha, j, s5);
    if (rc != SPS_OK && rc != SPS_ERR_NOT_CONVERGED) return rc;
    if (rc) r.worst = rc;
    if (st) st->mvops += 1;
    std::swap(ctx->d_gam, ctx->d_gam_new);
    std::swap(ctx->d_g, ctx->d_g_new);
    r.iters = j;
    r.best_iter = j;
    r.phi = std::sqrt(s5[0]);
    if (r.phi < tol) return SPS_OK;
    if (aux && r.phi < best_phi) {
      best_phi = r.phi;
      best_j = j;
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_gam_best, ctx->d_gam, sizeof(double) * nc,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_aux_best, aux, sizeof(double) * aux_len,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (!(r.phi < phi_limit)) return fail(SPS_ERR_BREAKDOWN, j);
    // BB1 throughout (variant 1), BB2 throughout (2), or BB1 on odd and BB2 on
    // even steps (3)
    const bool bb1 = ctx->prm.bb_variant == 1 || (ctx->prm.bb_variant == 3 && (j & 1));
    const bool ok = bb1 ? (s5[2] > 0) : (s5[2] > 0 && s5[3] > 0);
    if (!ok) {
      // s^T y <= 0: Algorithm 1 defines no step; stop, or keep the previous one
      if (!ctx->prm.bb_safeguard) return fail(SPS_ERR_BREAKDOWN, j);
      if (st) st->bb_safeguards += 1;
    } else {
      alpha = bb1 ? s5[1] / s5[2] : s5[2] / s5[3];
      ctx->bb_alpha_last = alpha;
    }
  }
  return fail(SPS_ERR_NOT_CONVERGED, j - 1);
}

// ---------------------------------------------------------------------------
// APGD (Sec. 3.3.1's comparison method): Nesterov's accelerated projected
// gradient with an adaptive Lipschitz estimate L (Mazhar et al. 2015).  Per
// iteration: M y at the extrapolated point, then x = max(y - g(y)/L, 0) and
// M x, with L doubled until the sufficient-decrease test, written for the
// quadratic objective as d.M d <= L |d|^2 (d = x - y), holds; the min-map
// residual of x decides convergence; the momentum restarts when
// g(x).(x - gamma) > 0; L shrinks by 0.9 after each accepted step.
// ---------------------------------------------------------------------------
constexpr int kApBlocks = 256;
__global__ void k_fill(int n, double v, double* __restrict__ out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) out[l] = v;
}
__global__ void k_apgd_step(int n, double t, const double* __restrict__ y, const double* __restrict__ My,
                            const double* __restrict__ q, double* __restrict__ x) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) x[l] = fmax(y[l] - t * (My[l] + q[l]), 0.0);
}
__global__ void k_apgd_extrap(int n, double beta, const double* __restrict__ x, const double* __restrict__ gam,
                              double* __restrict__ y) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) y[l] = x[l] + beta * (x[l] - gam[l]);
}
// per-block partials of [sum min(x, gx)^2, (x - gam).gx, (x - y).(Mx - My), |x - y|^2]
__global__ void __launch_bounds__(256) k_apgd_stats(int n, const double* __restrict__ x, const double* __restrict__ y,
                                                    const double* __restrict__ Mx, const double* __restrict__ My,
                                                    const double* __restrict__ q, const double* __restrict__ gam,
                                                    double* __restrict__ part) {
  __shared__ double sh[4][256];
  double a[4] = {0, 0, 0, 0};
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
    const double gx = Mx[l] + q[l], d = x[l] - y[l], mn = fmin(x[l], gx);
    a[0] = fma(mn, mn, a[0]);
    a[1] = fma(x[l] - gam[l], gx, a[1]);
    a[2] = fma(d, Mx[l] - My[l], a[2]);
    a[3] = fma(d, d, a[3]);
  }
  for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = a[c];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; ++c) part[c * kApBlocks + blockIdx.x] = sh[c][0];
}
__global__ void k_apgd_finish(const double* __restrict__ part, double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= 4) return;
  double s = 0.0;
  for (int b = 0; b < kApBlocks; ++b) s += part[c * kApBlocks + b];
  out[c] = s;
}

// mul(v, out): out = M v, one evaluation of M (a mobility solve for the
// boundary-integral mobility) leaving M D v in aux when aux is not null.
// On return d_gam holds the returned iterate and aux its M D gamma.
template <class Mul>
static int apgd_run(sps_ctx* ctx, int nc, sps_stats* st, Mul mul, BBResult& r, double* aux, size_t aux_len) {
  const int tb = (nc + 255) / 256;
  SPS_TRY(sps_grow(ctx, &ctx->d_apgd, ctx->cap_apgd, 3 * (size_t)nc + 8 * kApBlocks + 8));
  double* y = ctx->d_apgd;
  double* My = y + nc;
  double* tmp = My + nc;
  double* part = tmp + nc;
  double* res = part + 4 * kApBlocks;
  double* x = ctx->d_gam_new;
  double* Mx = ctx->d_Mg;
  if (aux) SPS_TRY(sps_grow(ctx, &ctx->d_aux_best, ctx->cap_aux_best, std::max<size_t>(aux_len, 1)));
  int rc = SPS_OK;
  auto note = [&](int rc2) -> int {
    if (rc2 != SPS_OK && rc2 != SPS_ERR_NOT_CONVERGED) return rc2;
    if (rc2) r.worst = rc2;
    if (st) st->mvops += 1;
    return SPS_OK;
  };
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_gam, 0, sizeof(double) * nc, ctx->stream));
  SPS_CUDA(ctx, cudaMemsetAsync(y, 0, sizeof(double) * nc, ctx->stream));
  SPS_CUDA(ctx, cudaMemsetAsync(My, 0, sizeof(double) * nc, ctx->stream));
  if (aux) SPS_CUDA(ctx, cudaMemsetAsync(aux, 0, sizeof(double) * aux_len, ctx->stream));
  // gamma_0 = 0: residual |min(0, q)|
  double s5[5];
  SPS_TRY(bb_stats(ctx, ctx->d_gam, ctx->d_q, nullptr, nullptr, s5));
  r.phi = std::sqrt(s5[0]);
  const double tol = ctx->prm.bbpgd_tol;
  if (r.phi < tol) return SPS_OK;
  // L_0 = |M e| / |e| for the vector of ones e
  k_fill<<<tb, 256, 0, ctx->stream>>>(nc, 1.0, tmp);
  SPS_LAUNCHED(ctx);
  SPS_TRY(note(mul(tmp, Mx)));
  double mm = 0.0;
  SPS_TRY(sps_dot(ctx, Mx, Mx, nc, &mm));
  double L = std::sqrt(mm / nc);
  if (!(L > 0) || !std::isfinite(L)) {
    r.bb_rc = SPS_ERR_BREAKDOWN;
    return SPS_OK;
  }
  double theta = 1.0;
  bool y_zero = true, y_known = false;   // M y already in My (y = 0, or a restart at x)
  double st4[4] = {0, 0, 0, 0};
  for (int k = 1; k <= ctx->prm.bbpgd_max; ++k) {
    if (!y_zero && !y_known) SPS_TRY(note(mul(y, My)));
    y_known = false;
    bool accepted = false;
    for (int bt = 0; bt < 64 && !accepted; ++bt) {
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_apgd_step<<<tb, 256, 0, ctx->stream>>>(nc, 1.0 / L, y, My, ctx->d_q, x); }
      SPS_LAUNCHED(ctx);
      SPS_TRY(note(mul(x, Mx)));
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_apgd_stats<<<kApBlocks, 256, 0, ctx->stream>>>(nc, x, y, Mx, My, ctx->d_q, ctx->d_gam, part);
      k_apgd_finish<<<1, 32, 0, ctx->stream>>>(part, res); }
      SPS_LAUNCHED(ctx);
      SPS_TRY(to_host(ctx, res, 4, st4));
      for (int c = 0; c < 4; ++c)
        if (!std::isfinite(st4[c])) return sps_fail(ctx, SPS_ERR_NONFINITE, "APGD: non-finite residual");
      if (st4[2] <= L * st4[3]) accepted = true;
      else L *= 2.0;
    }
    if (!accepted) {
      r.bb_rc = SPS_ERR_BREAKDOWN;    // no step length satisfied the decrease test
      return SPS_OK;
    }
    r.iters = k;
    r.best_iter = k;
    r.phi = std::sqrt(st4[0]);
    const bool restart = st4[1] > 0;
    // gamma <- x (its M D x is in aux)
    std::swap(ctx->d_gam, ctx->d_gam_new);
    x = ctx->d_gam_new;
    if (aux) SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_aux_best, aux, sizeof(double) * aux_len, cudaMemcpyDeviceToDevice,
                                           ctx->stream));
    if (r.phi < tol) break;
    if (k == ctx->prm.bbpgd_max) {
      r.bb_rc = SPS_ERR_NOT_CONVERGED;
      break;
    }
    const double th2 = theta * theta;
    double theta_new = 0.5 * (-th2 + theta * std::sqrt(th2 + 4.0));
    const double beta = theta * (1.0 - theta) / (th2 + theta_new);
    if (restart) {
      // y = gamma_k, whose product M gamma_k is the accepted M x
      SPS_CUDA(ctx, cudaMemcpyAsync(y, ctx->d_gam, sizeof(double) * nc, cudaMemcpyDeviceToDevice, ctx->stream));
      SPS_CUDA(ctx, cudaMemcpyAsync(My, Mx, sizeof(double) * nc, cudaMemcpyDeviceToDevice, ctx->stream));
      theta_new = 1.0;
      y_known = true;
    } else {
      // y = gamma_k + beta (gamma_k - gamma_{k-1}); gamma_{k-1} is in x's buffer now
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_apgd_extrap<<<tb, 256, 0, ctx->stream>>>(nc, beta, ctx->d_gam, x, y); }
      SPS_LAUNCHED(ctx);
    }
    y_zero = false;
    theta = theta_new;
    L *= 0.9;
  }
  if (aux) SPS_CUDA(ctx, cudaMemcpyAsync(aux, ctx->d_aux_best, sizeof(double) * aux_len, cudaMemcpyDeviceToDevice,
                                         ctx->stream));
  return rc;
}

static int finish_bb_stats(sps_ctx* ctx, int nc, const BBResult& r, sps_stats* st) {
  if (!st) return SPS_OK;
  st->bbpgd_iters = r.iters;
  st->final_phi = r.phi;
  if (nc > 0) SPS_TRY(sps_count_positive(ctx, ctx->d_gam, nc, &st->n_active));
  return SPS_OK;
}

// ---------------------------------------------------------------------------
// Minimum-map Newton (Sec. 3.3.1's second-order comparison method, after
// Niebe and Erleben 2015): Newton steps on H(gamma) = min(gamma, g),
// g = M gamma + q.  The Jacobian takes row l of M where g_l < gamma_l (the set
// F) and row l of the identity elsewhere, so Delta_l = -gamma_l off F and
// M_FF Delta_F = -(g + M [0; Delta_off F])_F, solved by conjugate gradients
// from 0 to relative residual kNtCgTol; M Delta is the CG-weighted sum of the
// products, so every line-search trial is free of products.  Step t = 1,
// halved until |H(gamma + t Delta)|^2 <= (1 - 2 sigma t) |H(gamma)|^2.
// ---------------------------------------------------------------------------
constexpr double kNtCgTol = 1e-3, kNtSigma = 1e-4;
constexpr int kNtCgMax = 200, kNtHalvings = 30;

__device__ __forceinline__ bool nt_free(const double* gam, const double* g, int l) { return g[l] < gam[l]; }

// dC = -gamma off F, 0 on F
__global__ void k_nt_offset(int n, const double* __restrict__ gam, const double* __restrict__ g,
                            double* __restrict__ dC) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) dC[l] = nt_free(gam, g, l) ? 0.0 : -gam[l];
}
// r = p = -(g + M dC) on F, 0 elsewhere; x = M x_F = 0
__global__ void k_nt_rhs(int n, const double* __restrict__ gam, const double* __restrict__ g,
                         const double* __restrict__ MdC, double* __restrict__ r, double* __restrict__ pd,
                         double* __restrict__ x, double* __restrict__ MxF) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const double v = nt_free(gam, g, l) ? -g[l] - MdC[l] : 0.0;
  r[l] = v;
  pd[l] = v;
  x[l] = 0.0;
  MxF[l] = 0.0;
}
// x += a p, M x_F += a M p, r -= a (M p restricted to F)
__global__ void k_nt_cg(int n, double a, const double* __restrict__ gam, const double* __restrict__ g,
                        const double* __restrict__ pd, const double* __restrict__ Mp, double* __restrict__ x,
                        double* __restrict__ MxF, double* __restrict__ r) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  x[l] += a * pd[l];
  MxF[l] += a * Mp[l];
  if (nt_free(gam, g, l)) r[l] -= a * Mp[l];
}
__global__ void k_nt_dir(int n, double b, const double* __restrict__ r, double* __restrict__ pd) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) pd[l] = r[l] + b * pd[l];
}
// Delta = x + dC, M Delta = M x_F + M dC (in place of x and M x_F)
__global__ void k_nt_step(int n, const double* __restrict__ dC, const double* __restrict__ MdC,
                          double* __restrict__ d, double* __restrict__ Md) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  d[l] += dC[l];
  Md[l] += MdC[l];
}
// partials of |min(gamma + t Delta, g + t M Delta)|^2 (slot 0 of the APGD layout)
__global__ void __launch_bounds__(256) k_nt_merit(int n, double t, const double* __restrict__ gam,
                                                  const double* __restrict__ g, const double* __restrict__ d,
                                                  const double* __restrict__ Md, double* __restrict__ part) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
    const double mn = fmin(fma(t, d[l], gam[l]), fma(t, Md[l], g[l]));
    a = fma(mn, mn, a);
  }
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sh[0];
    for (int c = 1; c < 4; ++c) part[c * kApBlocks + blockIdx.x] = 0.0;
  }
}
__global__ void k_nt_accept(int n, double t, double* __restrict__ gam, double* __restrict__ g,
                            const double* __restrict__ d, const double* __restrict__ Md) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  gam[l] = fma(t, d[l], gam[l]);
  g[l] = fma(t, Md[l], g[l]);
}

// mul(v, out): out = M v.  From gamma_0 = 0; on return d_gam / d_g hold the
// last accepted iterate and its g.
template <class Mul>
static int newton_run(sps_ctx* ctx, int nc, sps_stats* st, Mul mul, BBResult& r) {
  const int tb = (nc + 255) / 256;
  SPS_TRY(sps_grow(ctx, &ctx->d_apgd, ctx->cap_apgd, 7 * (size_t)nc + 8 * kApBlocks + 8));
  double* dC = ctx->d_apgd;
  double* MdC = dC + nc;
  double* x = MdC + nc;      // becomes Delta
  double* MxF = x + nc;      // becomes M Delta
  double* rv = MxF + nc;
  double* pd = rv + nc;
  double* Mp = pd + nc;
  double* part = Mp + nc;
  double* res = part + 4 * kApBlocks;
  double* gam = ctx->d_gam;
  double* g = ctx->d_g;
  auto note = [&](int rc2) -> int {
    if (rc2 != SPS_OK && rc2 != SPS_ERR_NOT_CONVERGED) return rc2;
    if (rc2) r.worst = rc2;
    if (st) st->mvops += 1;
    return SPS_OK;
  };
  SPS_CUDA(ctx, cudaMemsetAsync(gam, 0, sizeof(double) * nc, ctx->stream));
  SPS_CUDA(ctx, cudaMemcpyAsync(g, ctx->d_q, sizeof(double) * nc, cudaMemcpyDeviceToDevice, ctx->stream));
  double s5[5];
  SPS_TRY(bb_stats(ctx, gam, g, nullptr, nullptr, s5));
  double phi = std::sqrt(s5[0]);
  r.phi = phi;
  const double tol = ctx->prm.bbpgd_tol;
  if (phi < tol) return SPS_OK;
  for (int k = 1; k <= ctx->prm.bbpgd_max; ++k) {
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_nt_offset<<<tb, 256, 0, ctx->stream>>>(nc, gam, g, dC); }
    SPS_LAUNCHED(ctx);
    double cc = 0.0;
    SPS_TRY(sps_dot(ctx, dC, dC, nc, &cc));
    if (cc > 0) SPS_TRY(note(mul(dC, MdC)));
    else SPS_CUDA(ctx, cudaMemsetAsync(MdC, 0, sizeof(double) * nc, ctx->stream));
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_nt_rhs<<<tb, 256, 0, ctx->stream>>>(nc, gam, g, MdC, rv, pd, x, MxF); }
    SPS_LAUNCHED(ctx);
    double rr = 0.0;
    SPS_TRY(sps_dot(ctx, rv, rv, nc, &rr));
    const double bnorm = std::sqrt(rr);
    for (int it = 0; it < kNtCgMax; ++it) {
      if (std::sqrt(rr) <= kNtCgTol * bnorm) break;
      SPS_TRY(note(mul(pd, Mp)));
      double pAp = 0.0;   // p vanishes off F, so p . M p = p . (M p)_F
      SPS_TRY(sps_dot(ctx, pd, Mp, nc, &pAp));
      if (!(pAp > 0)) break;
      const double a = rr / pAp;
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_nt_cg<<<tb, 256, 0, ctx->stream>>>(nc, a, gam, g, pd, Mp, x, MxF, rv); }
      SPS_LAUNCHED(ctx);
      double rr_new = 0.0;
      SPS_TRY(sps_dot(ctx, rv, rv, nc, &rr_new));
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_nt_dir<<<tb, 256, 0, ctx->stream>>>(nc, rr_new / rr, rv, pd); }
      SPS_LAUNCHED(ctx);
      rr = rr_new;
    }
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_nt_step<<<tb, 256, 0, ctx->stream>>>(nc, dC, MdC, x, MxF); }
    SPS_LAUNCHED(ctx);
    const double theta0 = 0.5 * phi * phi;
    double t = 1.0, phi_t = 0.0;
    bool accepted = false;
    for (int h = 0; h <= kNtHalvings; ++h) {
      double st4[4];
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_nt_merit<<<kApBlocks, 256, 0, ctx->stream>>>(nc, t, gam, g, x, MxF, part);
      k_apgd_finish<<<1, 32, 0, ctx->stream>>>(part, res); }
      SPS_LAUNCHED(ctx);
      SPS_TRY(to_host(ctx, res, 4, st4));
      if (!std::isfinite(st4[0])) return sps_fail(ctx, SPS_ERR_NONFINITE, "Newton: non-finite residual");
      phi_t = std::sqrt(st4[0]);
      if (0.5 * st4[0] <= (1.0 - 2.0 * kNtSigma * t) * theta0) {
        accepted = true;
        break;
      }
      t *= 0.5;
    }
    if (!accepted) {
      r.bb_rc = SPS_ERR_BREAKDOWN;   // no step length met the Armijo test
      return SPS_OK;
    }
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_nt_accept<<<tb, 256, 0, ctx->stream>>>(nc, t, gam, g, x, MxF); }
    SPS_LAUNCHED(ctx);
    phi = phi_t;
    r.iters = k;
    r.best_iter = k;
    r.phi = phi;
    if (phi < tol) return SPS_OK;
  }
  r.bb_rc = SPS_ERR_NOT_CONVERGED;
  return SPS_OK;
}

static int resolve(sps_ctx* ctx, int n, const double* pos, const double* radii, const double* FT_ext,
                   double dt, double* gamma, int gamma_cap, double* UO, double* pos_out, sps_stats* st) {
  if (!(dt > 0)) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "dt must be positive");
  SPS_TRY(sps_set_geometry(ctx, n, pos, radii));
  SPS_TRY(check_finite_host(ctx, FT_ext, 6LL * n, "external force/torque"));
  ProjScope proj_scope(ctx);
  // 1. U_nc (warm start from the previous step's density when the size matches)
  const bool warm_nc = ctx->prm.warm_start && ctx->zeta_nc_n == ctx->NP;
  int rc = mobility_solve(ctx, FT_ext, ctx->d_Unc, st, ctx->d_zeta_nc, warm_nc);
  ctx->zeta_nc_n = (rc == SPS_OK) ? ctx->NP : 0;
  if (rc != SPS_OK && rc != SPS_ERR_NOT_CONVERGED) return rc;
  int worst = rc;
  // 2. contacts and D
  SPS_TRY(sps_launch_contacts(ctx, n, ctx->d_pos, ctx->d_rad));
  ctx->c_N = n;
  const int nc = ctx->n_c;
  if (st) st->n_contacts = nc;
  if (nc > gamma_cap) return sps_fail(ctx, SPS_ERR_CAPACITY, "gamma capacity smaller than the contact count");
  SPS_TRY(ensure_bb(ctx, nc));
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_Uc, 0, sizeof(double) * 6 * n, ctx->stream));
  BBResult r;
  if (nc > 0) {
    // 3. q = Phi/dt + D^T U_nc; BBPGD (Algorithm 1) from gamma_0 = 0 or, with
    //    bb_warm, from the previous step's gamma
    SPS_TRY(sps_launch_DT(ctx, ctx->d_Unc, ctx->d_q));
    const int tb = (nc + 255) / 256;
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_q<<<tb, 256, 0, ctx->stream>>>(nc, ctx->d_cphi, 1.0 / dt, ctx->d_q); }
    SPS_LAUNCHED(ctx);
    auto mul_g = [&]() { return apply_M(ctx, ctx->d_g, ctx->d_Mg, st, false); };
    auto step = [&](double alpha, int j, double s5[5]) -> int {
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_bb_step<<<tb, 256, 0, ctx->stream>>>(nc, alpha, ctx->d_gam, ctx->d_g, ctx->d_gam_new); }
      SPS_LAUNCHED(ctx);
      const int rc2 = apply_M(ctx, ctx->d_gam_new, ctx->d_Mg, st, ctx->prm.warm_start && j >= 2);
      if (rc2 != SPS_OK && rc2 != SPS_ERR_NOT_CONVERGED) return rc2;
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_add<<<tb, 256, 0, ctx->stream>>>(nc, ctx->d_Mg, ctx->d_q, ctx->d_g_new); }
      SPS_LAUNCHED(ctx);
      SPS_TRY(bb_stats(ctx, ctx->d_gam_new, ctx->d_g_new, ctx->d_gam, ctx->d_g, s5));
      return rc2;
    };
    // gamma_0: the previous step's gamma on the shared pairs (bb_warm), else 0
    bool warm0 = false;
    if (ctx->prm.bb_warm && ctx->prev_nc > 0 && ctx->prev_N == n) {
      { SpsPhase timer_(ctx, SPS_PH_BBPGD);
      k_map_gamma<<<tb, 256, 0, ctx->stream>>>(nc, ctx->d_cij, ctx->n_pair, ctx->prev_nc, ctx->prev_npair,
                                               ctx->d_prev_ij,
                                               ctx->d_prev_gam, ctx->d_gam); }
      SPS_LAUNCHED(ctx);
      int npos = 0;
      SPS_TRY(sps_count_positive(ctx, ctx->d_gam, nc, &npos));
      warm0 = npos > 0;
    }
    auto mul_gam = [&]() { return apply_M(ctx, ctx->d_gam, ctx->d_Mg, st, false); };
    if (ctx->prm.lcp_solver == 1) {
      auto mul = [&](const double* v, double* out) { return apply_M(ctx, v, out, st, ctx->prm.warm_start != 0); };
      SPS_TRY(apgd_run(ctx, nc, st, mul, r, ctx->d_Uc, 6 * (size_t)n));
      warm0 = true;   // (U_c below is the solve of the returned iterate, also at iteration 0)
    } else if (ctx->prm.lcp_solver == 2) {
      // products of CG directions: no useful warm start between them
      auto mul = [&](const double* v, double* out) { return apply_M(ctx, v, out, st, false); };
      SPS_TRY(newton_run(ctx, nc, st, mul, r));
      warm0 = false;
      if (r.iters > 0) {
        // U_c of the returned iterate: one more solve, M D gamma in d_Uc
        const int rc2 = apply_M(ctx, ctx->d_gam, ctx->d_Mg, st, false);
        if (rc2 != SPS_OK && rc2 != SPS_ERR_NOT_CONVERGED) return rc2;
        if (rc2) r.worst = rc2;
      }
    } else {
      SPS_TRY(bbpgd_run(ctx, nc, st, mul_g, step, r, ctx->d_Uc, 6 * (size_t)n, warm0, mul_gam));
    }
    if (r.worst) worst = r.worst;
    // U_c is the solve of the returned iterate; gamma_0 = 0 needs none
    if (r.iters == 0 && !warm0)
      SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_Uc, 0, sizeof(double) * 6 * n, ctx->stream));
    if (gamma)
      SPS_CUDA(ctx, cudaMemcpyAsync(gamma, ctx->d_gam, sizeof(double) * nc, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  // this step's pairs and gamma: the next step's initial guess (bb_warm = 2:
  // with the last step length of a converged Algorithm 1)
  ctx->prev_nc = 0;
  ctx->prev_alpha = (ctx->prm.lcp_solver == 0 && r.bb_rc == SPS_OK && r.iters > 0) ? ctx->bb_alpha_last : 0.0;
  if (ctx->prm.bb_warm && nc > 0) {
    SPS_TRY(sps_grow(ctx, &ctx->d_prev_ij, ctx->cap_prev_ij, 2 * (size_t)nc));
    SPS_TRY(sps_grow(ctx, &ctx->d_prev_gam, ctx->cap_prev_gam, (size_t)nc));
    SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_prev_ij, ctx->d_cij, sizeof(int) * 2 * nc, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_prev_gam, ctx->d_gam, sizeof(double) * nc, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    ctx->prev_nc = nc;
    ctx->prev_npair = ctx->n_pair;
  }
  ctx->prev_N = n;
  SPS_TRY(finish_bb_stats(ctx, nc, r, st));
  // 4. U = U_nc + U_c, pos += U dt
  const long long n6 = 6LL * n;
  { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
  k_axpby<<<gblocks(n6), 256, 0, ctx->stream>>>(n6, 1.0, ctx->d_Unc, 1.0, ctx->d_Uc, UO); }
  SPS_LAUNCHED(ctx);
  if (pos_out) {
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_pos_update<<<(3 * n + 255) / 256, 256, 0, ctx->stream>>>(n, pos, UO, dt, pos_out); }
    SPS_LAUNCHED(ctx);
  }
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (r.bb_rc != SPS_OK)
    return sps_fail(ctx, r.bb_rc, r.bb_rc == SPS_ERR_BREAKDOWN ? "BBPGD breakdown" : "BBPGD not converged");
  if (worst != SPS_OK) return sps_fail(ctx, worst, "a mobility solve did not converge");
  return SPS_OK;
}

static int ensure_ident(sps_ctx* ctx, int n) {
  if ((size_t)n <= ctx->cap_ident && ctx->d_F3) return SPS_OK;
  cudaFree(ctx->d_F3);
  cudaFree(ctx->d_iFT);
  ctx->d_F3 = ctx->d_iFT = nullptr;
  size_t c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_F3, c, 3 * (size_t)n));
  c = 0;
  SPS_TRY(sps_grow(ctx, &ctx->d_iFT, c, 6 * (size_t)n));
  ctx->cap_ident = n;
  return SPS_OK;
}

// The same step with the identity mobility (U = F): U_nc = F_ext, M = D^T D,
// and each BBPGD iteration is two fused passes (per sphere: projected step
// and D; per contact: D^T, + q and the statistics).  No surface grid exists.
static int resolve_identity(sps_ctx* ctx, int n, const double* pos, const double* radii,
                            const double* FT_ext, double dt, double* gamma, int gamma_cap, double* UO,
                            double* pos_out, sps_stats* st) {
  if (!(dt > 0)) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "dt must be positive");
  SPS_TRY(sps_check_inputs(ctx, n, pos, radii, FT_ext));
  SPS_TRY(ensure_ident(ctx, n));
  SPS_TRY(sps_launch_contacts(ctx, n, pos, radii));
  ctx->c_N = n;
  const int nc = ctx->n_c;
  if (st) st->n_contacts = nc;
  if (nc > gamma_cap) return sps_fail(ctx, SPS_ERR_CAPACITY, "gamma capacity smaller than the contact count");
  SPS_TRY(ensure_bb(ctx, nc));
  BBResult r;
  if (nc > 0) {
    SPS_TRY(sps_launch_DT(ctx, FT_ext, ctx->d_q));
    const int tb = (nc + 255) / 256;
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_q<<<tb, 256, 0, ctx->stream>>>(nc, ctx->d_cphi, 1.0 / dt, ctx->d_q); }
    SPS_LAUNCHED(ctx);
    auto mul_g = [&]() -> int {
      SPS_TRY(sps_launch_D(ctx, ctx->d_g, ctx->d_iFT));
      return sps_launch_DT(ctx, ctx->d_iFT, ctx->d_Mg);
    };
    auto step = [&](double alpha, int, double s5[5]) -> int {
      SPS_TRY(sps_launch_bb_identity(ctx, alpha, ctx->d_gam, ctx->d_g, ctx->d_gam_new, ctx->d_g_new));
      return read5(ctx, s5);
    };
    if (ctx->prm.lcp_solver != 0) {
      auto mul = [&](const double* v, double* out) -> int {
        SPS_TRY(sps_launch_D(ctx, v, ctx->d_iFT));
        return sps_launch_DT(ctx, ctx->d_iFT, out);
      };
      if (ctx->prm.lcp_solver == 1) SPS_TRY(apgd_run(ctx, nc, st, mul, r, nullptr, 0));
      else SPS_TRY(newton_run(ctx, nc, st, mul, r));
    } else {
      SPS_TRY(bbpgd_run(ctx, nc, st, mul_g, step, r, nullptr, 0, false, []() { return SPS_OK; }));
    }
    if (gamma)
      SPS_CUDA(ctx, cudaMemcpyAsync(gamma, ctx->d_gam, sizeof(double) * nc, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  SPS_TRY(finish_bb_stats(ctx, nc, r, st));
  // U = F_ext + D gamma (d_F3 holds D of the returned iterate after a BBPGD step)
  if (ctx->prm.lcp_solver != 0 && nc > 0) {
    SPS_TRY(sps_launch_D(ctx, ctx->d_gam, ctx->d_iFT));
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_axpby<<<gblocks(6LL * n), 256, 0, ctx->stream>>>(6LL * n, 1.0, FT_ext, 1.0, ctx->d_iFT, UO); }
    SPS_LAUNCHED(ctx);
  } else {
    SPS_TRY(sps_launch_identity_U(ctx, n, FT_ext, r.iters > 0 ? ctx->d_F3 : nullptr, UO));
  }
  if (pos_out) {
    { SpsPhase timer_(ctx, SPS_PH_BBPGD);
    k_pos_update<<<(3 * n + 255) / 256, 256, 0, ctx->stream>>>(n, pos, UO, dt, pos_out); }
    SPS_LAUNCHED(ctx);
  }
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (r.bb_rc != SPS_OK)
    return sps_fail(ctx, r.bb_rc, r.bb_rc == SPS_ERR_BREAKDOWN ? "BBPGD breakdown" : "BBPGD not converged");
  return SPS_OK;
}

static int resolve_any(sps_ctx* ctx, int n, const double* pos, const double* radii, const double* FT_ext,
                       double dt, double* gamma, int gamma_cap, double* UO, double* pos_out, sps_stats* st) {
  if (ctx->prm.mobility == SPS_MOB_IDENTITY)
    return resolve_identity(ctx, n, pos, radii, FT_ext, dt, gamma, gamma_cap, UO, pos_out, st);
  return resolve(ctx, n, pos, radii, FT_ext, dt, gamma, gamma_cap, UO, pos_out, st);
}

extern "C" int sps_resolve_collisions(sps_ctx* ctx, int n, const double* pos, const double* radii,
                                      const double* FT_ext, double dt, double* gamma, int gamma_cap,
                                      double* UO, double* pos_out, sps_stats* st) {
  if (!ctx || n < 1 || !pos || !radii || !FT_ext || !UO || gamma_cap < 0 || (gamma_cap > 0 && !gamma))
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "resolve_collisions: bad argument");
  long long l0;
  stats_begin(ctx, st, &l0);
  const int rc = resolve_any(ctx, n, pos, radii, FT_ext, dt, gamma, gamma_cap, UO, pos_out, st);
  return stats_end(ctx, st, l0, rc);
}

extern "C" int sps_simulate(sps_ctx* ctx, int n, double* pos, const double* radii, const double* FT_ext,
                            double dt, int steps, double* UO, sps_stats* stats_per_step, int* steps_done) {
  if (!ctx || n < 1 || !pos || !radii || !FT_ext || !UO || steps < 0)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "simulate: bad argument");
  if (steps_done) *steps_done = 0;
  for (int k = 0; k < steps; ++k) {
    sps_stats tmp;
    sps_stats* st = stats_per_step ? stats_per_step + k : &tmp;
    long long l0;
    stats_begin(ctx, st, &l0);
    // positions advance in place: the step reads pos into the context before
    // its last kernel overwrites it element by element
    const int rc = stats_end(ctx, st, l0, resolve_any(ctx, n, pos, radii, FT_ext, dt, nullptr, INT32_MAX,
                                                      UO, pos, st));
    if (rc != SPS_OK) return rc;
    if (steps_done) *steps_done = k + 1;
  }
  return SPS_OK;
}

extern "C" int sps_resolve_collisions_host(sps_ctx* ctx, int n, const double* pos, const double* radii,
                                           const double* FT_ext, double dt, double* gamma, int gamma_cap,
                                           double* UO, double* pos_out, int* n_contacts_out,
                                           sps_stats* st) {
  if (!ctx || n < 1 || !pos || !radii || !FT_ext || !UO || gamma_cap < 0 || (gamma_cap > 0 && !gamma))
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "resolve_collisions_host: bad argument");
  // device staging: pos, radii, FT in, UO, pos_out, gamma out
  double *d = nullptr;
  const size_t need = 3 * (size_t)n + n + 6 * (size_t)n + 6 * (size_t)n + 3 * (size_t)n +
                      (size_t)std::max(gamma_cap, 1);
  SPS_CUDA(ctx, cudaMallocAsync((void**)&d, need * sizeof(double), ctx->stream));
  double *dp = d, *dr = dp + 3 * n, *dF = dr + n, *dU = dF + 6 * n, *dpo = dU + 6 * n, *dg = dpo + 3 * n;
  SPS_CUDA(ctx, cudaMemcpyAsync(dp, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
  SPS_CUDA(ctx, cudaMemcpyAsync(dr, radii, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  SPS_CUDA(ctx, cudaMemcpyAsync(dF, FT_ext, sizeof(double) * 6 * n, cudaMemcpyHostToDevice, ctx->stream));
  long long l0;
  stats_begin(ctx, st, &l0);
  int rc = resolve_any(ctx, n, dp, dr, dF, dt, dg, gamma_cap, dU, pos_out ? dpo : nullptr, st);
  if (rc == SPS_OK || rc == SPS_ERR_NOT_CONVERGED || rc == SPS_ERR_BREAKDOWN) {
    cudaMemcpyAsync(UO, dU, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (pos_out) cudaMemcpyAsync(pos_out, dpo, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (ctx->n_c > 0 && ctx->n_c <= gamma_cap)
      cudaMemcpyAsync(gamma, dg, sizeof(double) * ctx->n_c, cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (n_contacts_out) *n_contacts_out = ctx->n_c;
  cudaFreeAsync(d, ctx->stream);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess && rc == SPS_OK) rc = sps_fail(ctx, SPS_ERR_CUDA, cudaGetErrorString(e));
  return stats_end(ctx, st, l0, rc);
}

// ---------------------------------------------------------------------------
// adjoint of the mobility solve (dL/dF; dL/dx in sps_adjoint_geom.cu)
// ---------------------------------------------------------------------------
int sps_geom_gradient(sps_ctx* ctx, const double* ubar, const double* lam, const double* sig, double* dx);

// out = M^T ubar (both N x 6) on the current geometry: the force/torque part of
// the adjoint of the mobility map.  ubar' = E^T ubar at the nodes (weights),
// s = S^T ubar', lambda = A^{-T} s (GMRES, cold start), rhobar = s -
// (I/2 + K)^T lambda, out = R^T rhobar.  Leaves ubar', lambda in d_ubar, d_lam.
static int mobility_T(sps_ctx* ctx, const double* ubar, double* out, sps_stats* st) {
  const long long n3 = 3LL * ctx->NP;
  SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_ubar, 0, sizeof(double) * n3, ctx->stream));
  SPS_TRY(sps_launch_add_L_w(ctx, ubar, ctx->d_ubar, true));
  SPS_TRY(sps_layer_T(ctx, SPS_OP_S, ctx->d_ubar, ctx->d_sbar));
  ctx->adjoint_mode = true;
  int its = 0;
  double res = 0.0;
  int grc = gmres(ctx, ctx->d_sbar, ctx->d_lam, false, ctx->prm.gmres_tol, ctx->prm.gmres_max, false, &its, &res);
  ctx->adjoint_mode = false;
  if (grc != SPS_OK && grc != SPS_ERR_NOT_CONVERGED) return grc;
  if (st) {
    st->mobility_solves += 1;
    st->gmres_iters += its;
    st->gmres_iters_max = std::max(st->gmres_iters_max, its);
    st->gmres_res_max = std::max(st->gmres_res_max, res);
  }
  SPS_TRY(sps_layer_T(ctx, SPS_OP_K, ctx->d_lam, ctx->d_rbar));
  { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
  k_combine3<<<gblocks(n3), 256, 0, ctx->stream>>>(n3, ctx->d_sbar, ctx->d_lam, ctx->d_rbar); }
  SPS_LAUNCHED(ctx);
  SPS_TRY(sps_launch_moments_w(ctx, ctx->d_rbar, ctx->d_mom, false));
  SPS_TRY(sps_launch_extract(ctx, ctx->d_mom, out));
  return grc;
}

extern "C" int sps_mobility_adjoint(sps_ctx* ctx, int n, const double* pos, const double* radii,
                                    const double* FT, const double* dL_dU, double* UO, double* dL_dFT,
                                    double* dL_dpos, sps_stats* st) {
  if (!ctx || !FT || !dL_dU || !dL_dFT || n < 1 || !pos || !radii)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "mobility_adjoint: bad argument");
  SPS_TRY(no_orientation(ctx, "mobility_adjoint"));
  long long l0;
  stats_begin(ctx, st, &l0);
  if (ctx->prm.mobility == SPS_MOB_IDENTITY) {
    // U = F: dL/dF = dL/dU, and U does not depend on the centres
    int rc = sps_check_inputs(ctx, n, pos, radii, FT);
    if (rc == SPS_OK) rc = sps_check_inputs(ctx, n, pos, radii, dL_dU);
    if (rc == SPS_OK && UO) rc = sps_launch_identity_U(ctx, n, FT, nullptr, UO);
    if (rc == SPS_OK) rc = sps_launch_identity_U(ctx, n, dL_dU, nullptr, dL_dFT);
    if (rc == SPS_OK && dL_dpos) {
      cudaError_t e = cudaMemsetAsync(dL_dpos, 0, sizeof(double) * 3 * n, ctx->stream);
      if (e != cudaSuccess) rc = sps_fail(ctx, SPS_ERR_CUDA, cudaGetErrorString(e));
    }
    if (rc == SPS_OK) {
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) rc = sps_fail(ctx, SPS_ERR_CUDA, cudaGetErrorString(e));
    }
    return stats_end(ctx, st, l0, rc);
  }
  int rc = sps_set_geometry(ctx, n, pos, radii);
  if (rc == SPS_OK) rc = check_finite_host(ctx, FT, 6LL * n, "force/torque");
  if (rc == SPS_OK) rc = check_finite_host(ctx, dL_dU, 6LL * n, "dL/dU");
  if (rc != SPS_OK) return stats_end(ctx, st, l0, rc);
  const long long n3 = 3LL * ctx->NP;
  // forward solve; keep sigma = rho + zeta
  double* U = UO ? UO : ctx->d_Uc;
  const bool warm = ctx->prm.warm_start && ctx->zeta_n == ctx->NP;
  int frc = mobility_solve(ctx, FT, U, st, ctx->d_zeta, warm);
  ctx->zeta_n = (frc == SPS_OK) ? ctx->NP : 0;
  if (frc != SPS_OK && frc != SPS_ERR_NOT_CONVERGED) return stats_end(ctx, st, l0, frc);
  SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_sigtot, ctx->d_tmp3, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                                ctx->stream));
  int grc = mobility_T(ctx, dL_dU, dL_dFT, st);
  if (grc != SPS_OK && grc != SPS_ERR_NOT_CONVERGED) return stats_end(ctx, st, l0, grc);
  if (dL_dpos) SPS_TRY(sps_geom_gradient(ctx, ctx->d_ubar, ctx->d_lam, ctx->d_sigtot, dL_dpos));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int out_rc = (frc != SPS_OK) ? frc : grc;
  return stats_end(ctx, st, l0, out_rc != SPS_OK ? sps_fail(ctx, out_rc, "adjoint: a solve did not converge") : SPS_OK);
}

// ---------------------------------------------------------------------------
// adjoint of the collision-resolved step in the external forces
// ---------------------------------------------------------------------------
// Applies M^T to an N x 6 force/torque array (identity: a copy).
static int apply_MT(sps_ctx* ctx, int n, const double* in, double* out, sps_stats* st) {
  if (ctx->prm.mobility == SPS_MOB_IDENTITY) {
    SPS_CUDA(ctx, cudaMemcpyAsync(out, in, sizeof(double) * 6 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return SPS_OK;
  }
  return mobility_T(ctx, in, out, st);
}

extern "C" int sps_collision_adjoint(sps_ctx* ctx, int n, const double* pos, const double* radii,
                                     const double* FT_ext, double dt, const double* dL_dU, double* UO,
                                     double* dL_dFT, double* dL_dpos, sps_stats* st) {
  if (!ctx || n < 1 || !pos || !radii || !FT_ext || !dL_dU || !UO || !dL_dFT)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "collision_adjoint: bad argument");
  SPS_TRY(no_orientation(ctx, "collision_adjoint"));
  if (ctx->walls.n > 0)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "collision_adjoint: not available with walls");
  long long l0;
  stats_begin(ctx, st, &l0);
  // forward step (positions are not advanced)
  int rc = resolve_any(ctx, n, pos, radii, FT_ext, dt, nullptr, INT32_MAX, UO, nullptr, st);
  if (rc != SPS_OK) return stats_end(ctx, st, l0, rc);
  const int nc = ctx->n_c;
  const size_t n6 = 6 * (size_t)n;
  size_t c = 0;
  if (ctx->cap_adj6 < n6) {
    cudaFree(ctx->d_adj6a);
    cudaFree(ctx->d_adj6b);
    ctx->d_adj6a = ctx->d_adj6b = nullptr;
    SPS_TRY(sps_grow(ctx, &ctx->d_adj6a, c, n6));
    c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_adj6b, c, n6));
    ctx->cap_adj6 = n6;
  }
  SPS_TRY(sps_grow(ctx, &ctx->d_adjc, ctx->cap_adjc, (size_t)std::max(nc, 1)));
  // v = M^T ubar: the gradient without contacts
  rc = apply_MT(ctx, n, dL_dU, dL_dFT, st);
  if (rc != SPS_OK && rc != SPS_ERR_NOT_CONVERGED) return stats_end(ctx, st, l0, rc);
  int worst = rc;
  std::vector<double> gam(nc);
  if (nc > 0) {
    SPS_CUDA(ctx, cudaMemcpyAsync(gam.data(), ctx->d_gam, sizeof(double) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  std::vector<char> act(nc);
  int na = 0;
  for (int l = 0; l < nc; ++l) na += (act[l] = gam[l] > 0.0);
  if (na > 0) {
    // matvec on contact vectors: y = P D^T M^T D P x + (I - P) x, P = diag(active)
    std::vector<double> xm(nc), y(nc);
    auto matvec = [&](const std::vector<double>& x, std::vector<double>& out) -> int {
      for (int l = 0; l < nc; ++l) xm[l] = act[l] ? x[l] : 0.0;
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_adjc, xm.data(), sizeof(double) * nc, cudaMemcpyHostToDevice,
                                    ctx->stream));
      SPS_TRY(sps_launch_D(ctx, ctx->d_adjc, ctx->d_adj6a));
      const int r2 = apply_MT(ctx, n, ctx->d_adj6a, ctx->d_adj6b, st);
      if (r2 != SPS_OK && r2 != SPS_ERR_NOT_CONVERGED) return r2;
      if (r2) worst = r2;
      SPS_TRY(sps_launch_DT(ctx, ctx->d_adj6b, ctx->d_adjc));
      SPS_CUDA(ctx, cudaMemcpyAsync(out.data(), ctx->d_adjc, sizeof(double) * nc, cudaMemcpyDeviceToHost,
                                    ctx->stream));
      SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      for (int l = 0; l < nc; ++l) out[l] = act[l] ? out[l] : x[l];
      return SPS_OK;
    };
    // right-hand side P D^T v
    std::vector<double> b(nc);
    SPS_TRY(sps_launch_DT(ctx, dL_dFT, ctx->d_adjc));
    SPS_CUDA(ctx, cudaMemcpyAsync(b.data(), ctx->d_adjc, sizeof(double) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int l = 0; l < nc; ++l) b[l] = act[l] ? b[l] : 0.0;
    // GMRES (modified Gram-Schmidt, x0 = 0) on the host: n_c-vectors are small
    const int kmax = ctx->prm.gmres_max;
    const double tol = ctx->prm.gmres_tol;
    double nb = 0.0;
    for (double v : b) nb += v * v;
    nb = std::sqrt(nb);
    std::vector<double> lam(nc, 0.0);
    if (nb > 0.0) {
      std::vector<std::vector<double>> V(1, b);
      for (double& v : V[0]) v /= nb;
      std::vector<double> H((size_t)(kmax + 1) * kmax, 0.0), cs(kmax), sn(kmax), g(kmax + 1, 0.0);
      auto Hc = [&](int r, int col) -> double& { return H[(size_t)col * (kmax + 1) + r]; };
      g[0] = nb;
      int k = 0;
      double res = 1.0;
      for (k = 1; k <= kmax; ++k) {
        std::vector<double> w(nc);
        rc = matvec(V[k - 1], w);
        if (rc != SPS_OK) return stats_end(ctx, st, l0, rc);
        for (int j = 0; j < k; ++j) {
          double h = 0.0;
          for (int l = 0; l < nc; ++l) h += V[j][l] * w[l];
          Hc(j, k - 1) = h;
          for (int l = 0; l < nc; ++l) w[l] -= h * V[j][l];
        }
        double hn = 0.0;
        for (double v : w) hn += v * v;
        hn = std::sqrt(hn);
        Hc(k, k - 1) = hn;
        for (int j = 0; j < k - 1; ++j) {
          const double a = Hc(j, k - 1), bq = Hc(j + 1, k - 1);
          Hc(j, k - 1) = cs[j] * a + sn[j] * bq;
          Hc(j + 1, k - 1) = -sn[j] * a + cs[j] * bq;
        }
        const double a = Hc(k - 1, k - 1), bq = Hc(k, k - 1);
        const double den = std::hypot(a, bq);
        if (!(den > 0.0)) {
          --k;
          break;
        }
        cs[k - 1] = a / den;
        sn[k - 1] = bq / den;
        Hc(k - 1, k - 1) = den;
        Hc(k, k - 1) = 0.0;
        g[k] = -sn[k - 1] * g[k - 1];
        g[k - 1] = cs[k - 1] * g[k - 1];
        res = std::fabs(g[k]) / nb;
        if (res < tol || hn == 0.0) break;
        for (double& v : w) v /= hn;
        V.push_back(std::move(w));
      }
      if (k > kmax) k = kmax;
      std::vector<double> yk(k);
      for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int j = i + 1; j < k; ++j) acc -= Hc(i, j) * yk[j];
        yk[i] = acc / Hc(i, i);
        if (!std::isfinite(yk[i]))
          return stats_end(ctx, st, l0, sps_fail(ctx, SPS_ERR_NONFINITE, "collision adjoint: singular system"));
      }
      for (int j = 0; j < k; ++j)
        for (int l = 0; l < nc; ++l) lam[l] += yk[j] * V[j][l];
      if (st) {
        st->gmres_res_max = std::max(st->gmres_res_max, res);
        st->ir_sweeps = k;    // outer (active-set) iterations
      }
      if (!(res < tol)) worst = SPS_ERR_NOT_CONVERGED;
    }
    // dL/dF = v - M^T D P lam
    for (int l = 0; l < nc; ++l) xm[l] = act[l] ? lam[l] : 0.0;
    SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_adjc, xm.data(), sizeof(double) * nc, cudaMemcpyHostToDevice,
                                  ctx->stream));
    SPS_TRY(sps_launch_D(ctx, ctx->d_adjc, ctx->d_adj6a));
    const int r3 = apply_MT(ctx, n, ctx->d_adj6a, ctx->d_adj6b, st);
    if (r3 != SPS_OK && r3 != SPS_ERR_NOT_CONVERGED) return stats_end(ctx, st, l0, r3);
    if (r3) worst = r3;
    { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
    k_axpby<<<gblocks((long long)n6), 256, 0, ctx->stream>>>((long long)n6, 1.0, dL_dFT, -1.0, ctx->d_adj6b,
                                                             dL_dFT); }
    SPS_LAUNCHED(ctx);
  }
  if (dL_dpos) {
    // dL/dc = (ubar - D_A mu)^T (dM/dc) F_tot + the contact-geometry terms,
    // mu = the active-set solution above (masked, in d_adjc), F_tot = F + D gamma
    const long long m6 = (long long)n6;
    if (na > 0) {
      SPS_TRY(sps_launch_D(ctx, ctx->d_adjc, ctx->d_adj6a));
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_axpby<<<gblocks(m6), 256, 0, ctx->stream>>>(m6, 1.0, dL_dU, -1.0, ctx->d_adj6a, ctx->d_adj6b); }
      SPS_LAUNCHED(ctx);
      SPS_TRY(sps_launch_D(ctx, ctx->d_gam, ctx->d_adj6a));
      { SpsPhase timer_(ctx, SPS_PH_KRYLOV);
      k_axpby<<<gblocks(m6), 256, 0, ctx->stream>>>(m6, 1.0, FT_ext, 1.0, ctx->d_adj6a, ctx->d_adj6a); }
      SPS_LAUNCHED(ctx);
    } else {
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_adj6b, dL_dU, sizeof(double) * n6, cudaMemcpyDeviceToDevice, ctx->stream));
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_adj6a, FT_ext, sizeof(double) * n6, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (ctx->prm.mobility == SPS_MOB_IDENTITY) {
      SPS_CUDA(ctx, cudaMemsetAsync(dL_dpos, 0, sizeof(double) * 3 * n, ctx->stream));
    } else {
      // forward solve with F_tot (keeps sigma), adjoint with a, then the
      // derivative of the far and near sums
      const long long n3 = 3LL * ctx->NP;
      int frc = mobility_solve(ctx, ctx->d_adj6a, ctx->d_Uc, st, ctx->d_zeta, false);
      ctx->zeta_n = 0;
      if (frc != SPS_OK && frc != SPS_ERR_NOT_CONVERGED) return stats_end(ctx, st, l0, frc);
      if (frc) worst = frc;
      SPS_CUDA(ctx, cudaMemcpyAsync(ctx->d_sigtot, ctx->d_tmp3, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
      int grc = mobility_T(ctx, ctx->d_adj6b, ctx->d_FT, st);
      if (grc != SPS_OK && grc != SPS_ERR_NOT_CONVERGED) return stats_end(ctx, st, l0, grc);
      if (grc) worst = grc;
      SPS_TRY(sps_geom_gradient(ctx, ctx->d_ubar, ctx->d_lam, ctx->d_sigtot, dL_dpos));
    }
    if (na > 0) SPS_TRY(sps_launch_contact_grad(ctx, pos, ctx->d_adjc, dL_dFT, UO, dt, dL_dpos));
  }
  if (st) st->n_active = na;
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (worst != SPS_OK) return stats_end(ctx, st, l0, sps_fail(ctx, worst, "collision adjoint: a solve did not converge"));
  return stats_end(ctx, st, l0, SPS_OK);
}
