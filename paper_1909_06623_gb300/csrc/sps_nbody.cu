// Far-field layer potentials by direct quadrature (Sec. 4.1 operators, Sec. 5.1
// "all-to-all" evaluation): for every target node x of sphere i and every
// source node y of a sphere j that is neither i nor a near neighbour of i,
//   S:  u(x) += w_y G(x-y) sigma(y),   G = (I/|r| + r r^T/|r|^3) / (8 pi)
//   K:  t(x) += w_y T(x-y) : sigma(y) n(x) = -3/(4 pi) w_y (r.sigma)(r.n) r/|r|^5
// (T is symmetric in its three indices).  Near and self pairs are skipped, not
// subtracted: their VSH values are added by the near / self kernels.
//
// FP64 kernel: one target per thread, source tiles staged in shared memory.
// FP32 kernel (mixed precision): two targets per thread, 256-source tiles in
// shared memory, rsqrt on the SFU, a warp-uniform fast path for tiles without
// excluded spheres, FP32 sums per tile combined with Kahan compensation across
// tiles, and a source split (gridDim.y) whose partial sums are added in FP64 in
// a fixed order.
#include "sps_internal.cuh"

namespace {

constexpr int kT64 = 128;   // FP64: targets per block == sources per tile

template <int OP>
__global__ void __launch_bounds__(kT64) k_far64(int N, int P, const double* __restrict__ X,
                                                const double* __restrict__ Nr,
                                                const double* __restrict__ W,
                                                const double* __restrict__ sig,
                                                const int* __restrict__ near_ptr,
                                                const int* __restrict__ near_idx,
                                                double* __restrict__ out) {
  __shared__ double sx[kT64], sy[kT64], sz[kT64], fx[kT64], fy[kT64], fz[kT64];
  __shared__ int ss[kT64];
  const long long NP = (long long)N * P;
  const long long t = (long long)blockIdx.x * kT64 + threadIdx.x;
  const bool valid = t < NP;
  const long long tt = valid ? t : 0;
  const double tx = X[tt], ty = X[NP + tt], tz = X[2 * NP + tt];
  double nx = 0, ny = 0, nz = 0;
  if (OP == SPS_OP_K) {
    nx = Nr[tt];
    ny = Nr[NP + tt];
    nz = Nr[2 * NP + tt];
  }
  const int i = (int)(tt / P);
  int ptr = near_ptr[i];
  const int end = near_ptr[i + 1];
  int cur = -1;
  bool excl = false;
  double ax = 0, ay = 0, az = 0;
  for (long long t0 = 0; t0 < NP; t0 += kT64) {
    const long long j = t0 + threadIdx.x;
    if (j < NP) {
      const double w = W[j];
      sx[threadIdx.x] = X[j];
      sy[threadIdx.x] = X[NP + j];
      sz[threadIdx.x] = X[2 * NP + j];
      fx[threadIdx.x] = w * sig[j];
      fy[threadIdx.x] = w * sig[NP + j];
      fz[threadIdx.x] = w * sig[2 * NP + j];
      ss[threadIdx.x] = (int)(j / P);
    }
    __syncthreads();
    const int nt = (int)min((long long)kT64, NP - t0);
    for (int k = 0; k < nt; ++k) {
      const int sj = ss[k];
      if (sj != cur) {
        cur = sj;
        while (ptr < end && near_idx[ptr] < sj) ++ptr;
        excl = (sj == i) || (ptr < end && near_idx[ptr] == sj);
      }
      if (excl) continue;
      const double rx = tx - sx[k], ry = ty - sy[k], rz = tz - sz[k];
      const double r2 = rx * rx + ry * ry + rz * rz;
      const double inv = rsqrt(r2);
      const double rs = rx * fx[k] + ry * fy[k] + rz * fz[k];
      if (OP == SPS_OP_S) {
        const double c = rs * inv * inv * inv;
        ax += fx[k] * inv + c * rx;
        ay += fy[k] * inv + c * ry;
        az += fz[k] * inv + c * rz;
      } else {
        const double rn = rx * nx + ry * ny + rz * nz;
        const double i2 = inv * inv;
        const double c = rs * rn * i2 * i2 * inv;
        ax += c * rx;
        ay += c * ry;
        az += c * rz;
      }
    }
    __syncthreads();
  }
  if (valid) {
    const double s = (OP == SPS_OP_S) ? 1.0 / (8.0 * SPS_PI) : -3.0 / (4.0 * SPS_PI);
    out[t] += s * ax;
    out[NP + t] += s * ay;
    out[2 * NP + t] += s * az;
  }
}

// ---------------------------------------------------------------------------
// FP32 kernel
// ---------------------------------------------------------------------------
constexpr int kT32 = 128;      // threads per block
constexpr int kTS32 = 256;     // sources per tile
constexpr int kTPT = 2;        // targets per thread

struct Excl {
  int i, ptr, end;
};

__device__ __forceinline__ unsigned long long excl_mask(Excl& e, const int* __restrict__ near_idx,
                                                        int s_lo, int s_hi) {
  unsigned long long m = 0ull;
  if (e.i >= s_lo && e.i <= s_hi) m |= 1ull << (e.i - s_lo);
  while (e.ptr < e.end && near_idx[e.ptr] < s_lo) ++e.ptr;
  for (int q = e.ptr; q < e.end; ++q) {
    const int s = near_idx[q];
    if (s > s_hi) break;
    m |= 1ull << (s - s_lo);
  }
  return m;
}

template <int OP>
__device__ __forceinline__ void pair32(float tx, float ty, float tz, float nx, float ny, float nz,
                                       const float4 a, const float4 b, float& ax, float& ay,
                                       float& az) {
  const float rx = tx - a.x, ry = ty - a.y, rz = tz - a.z;
  const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
  const float inv = rsqrtf(r2);
  const float rs = fmaf(rz, b.y, fmaf(ry, b.x, rx * a.w));
  if (OP == SPS_OP_S) {
    const float i2 = inv * inv;
    const float c = rs * i2 * inv;
    ax = fmaf(a.w, inv, fmaf(c, rx, ax));
    ay = fmaf(b.x, inv, fmaf(c, ry, ay));
    az = fmaf(b.y, inv, fmaf(c, rz, az));
  } else {
    const float rn = fmaf(rz, nz, fmaf(ry, ny, rx * nx));
    const float i2 = inv * inv;
    const float c = (rs * rn) * (i2 * i2 * inv);
    ax = fmaf(c, rx, ax);
    ay = fmaf(c, ry, ay);
    az = fmaf(c, rz, az);
  }
}

template <int OP>
__global__ void __launch_bounds__(kT32) k_far32(int N, int P, long long src_per_split,
                                                const float* __restrict__ X,
                                                const float* __restrict__ Nr,
                                                const float* __restrict__ W,
                                                const float* __restrict__ sig,
                                                const int* __restrict__ near_ptr,
                                                const int* __restrict__ near_idx,
                                                double* __restrict__ part) {
  __shared__ float4 sa[kTS32], sb[kTS32];
  __shared__ unsigned char sl[kTS32];
  const long long NP = (long long)N * P;
  const long long base = (long long)blockIdx.x * kT32 * kTPT + threadIdx.x;
  float tx[kTPT], ty[kTPT], tz[kTPT], nx[kTPT], ny[kTPT], nz[kTPT];
  float sx[kTPT], sy[kTPT], sz[kTPT], cx[kTPT], cy[kTPT], cz[kTPT];
  Excl ex[kTPT];
#pragma unroll
  for (int q = 0; q < kTPT; ++q) {
    const long long t = base + q * kT32;
    const long long tt = t < NP ? t : NP - 1;
    tx[q] = X[tt];
    ty[q] = X[NP + tt];
    tz[q] = X[2 * NP + tt];
    if (OP == SPS_OP_K) {
      nx[q] = Nr[tt];
      ny[q] = Nr[NP + tt];
      nz[q] = Nr[2 * NP + tt];
    } else {
      nx[q] = ny[q] = nz[q] = 0.f;
    }
    sx[q] = sy[q] = sz[q] = cx[q] = cy[q] = cz[q] = 0.f;
    ex[q].i = (int)(tt / P);
    ex[q].ptr = near_ptr[ex[q].i];
    ex[q].end = near_ptr[ex[q].i + 1];
  }
  const long long s0 = (long long)blockIdx.y * src_per_split;
  const long long s1 = min(NP, s0 + src_per_split);
  for (long long t0 = s0; t0 < s1; t0 += kTS32) {
    const int nt = (int)min((long long)kTS32, s1 - t0);
    const int s_lo = (int)(t0 / P), s_hi = (int)((t0 + nt - 1) / P);
    for (int k = threadIdx.x; k < kTS32; k += kT32) {
      const long long j = t0 + k;
      if (k < nt) {
        const float w = W[j];
        sa[k] = make_float4(X[j], X[NP + j], X[2 * NP + j], w * sig[j]);
        sb[k] = make_float4(w * sig[NP + j], w * sig[2 * NP + j], 0.f, 0.f);
        sl[k] = (unsigned char)(j / P - s_lo);
      } else {
        // padding sources far away with zero weight (never excluded)
        sa[k] = make_float4(1e18f, 1e18f, 1e18f, 0.f);
        sb[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        sl[k] = 63;
      }
    }
    __syncthreads();
    unsigned long long m[kTPT];
    bool any = false;
#pragma unroll
    for (int q = 0; q < kTPT; ++q) {
      m[q] = excl_mask(ex[q], near_idx, s_lo, s_hi);
      any |= (m[q] != 0ull);
    }
    float ax[kTPT], ay[kTPT], az[kTPT];
#pragma unroll
    for (int q = 0; q < kTPT; ++q) ax[q] = ay[q] = az[q] = 0.f;
    if (!__any_sync(0xffffffffu, any)) {
#pragma unroll 4
      for (int k = 0; k < kTS32; ++k) {
        const float4 a = sa[k], b = sb[k];
#pragma unroll
        for (int q = 0; q < kTPT; ++q)
          pair32<OP>(tx[q], ty[q], tz[q], nx[q], ny[q], nz[q], a, b, ax[q], ay[q], az[q]);
      }
    } else {
      for (int k = 0; k < kTS32; ++k) {
        const float4 a = sa[k], b = sb[k];
        const int l = sl[k];
#pragma unroll
        for (int q = 0; q < kTPT; ++q) {
          float bx = ax[q], by = ay[q], bz = az[q];
          pair32<OP>(tx[q], ty[q], tz[q], nx[q], ny[q], nz[q], a, b, bx, by, bz);
          const bool skip = (m[q] >> l) & 1ull;
          ax[q] = skip ? ax[q] : bx;
          ay[q] = skip ? ay[q] : by;
          az[q] = skip ? az[q] : bz;
        }
      }
    }
    // Kahan: fold this tile's FP32 sum into the running compensated sum
#pragma unroll
    for (int q = 0; q < kTPT; ++q) {
      float y, t;
      y = ax[q] - cx[q]; t = sx[q] + y; cx[q] = (t - sx[q]) - y; sx[q] = t;
      y = ay[q] - cy[q]; t = sy[q] + y; cy[q] = (t - sy[q]) - y; sy[q] = t;
      y = az[q] - cz[q]; t = sz[q] + y; cz[q] = (t - sz[q]) - y; sz[q] = t;
    }
    __syncthreads();
  }
  double* o = part + (long long)blockIdx.y * 3 * NP;
#pragma unroll
  for (int q = 0; q < kTPT; ++q) {
    const long long t = base + q * kT32;
    if (t < NP) {
      o[t] = (double)sx[q] - (double)cx[q];
      o[NP + t] = (double)sy[q] - (double)cy[q];
      o[2 * NP + t] = (double)sz[q] - (double)cz[q];
    }
  }
}

__global__ void k_reduce_parts(long long n3, int splits, const double* __restrict__ part,
                               double scale, double* __restrict__ out) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n3;
       g += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += part[k * n3 + g];
    out[g] += scale * s;
  }
}

__global__ void k_to_f32(long long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
       g += (long long)gridDim.x * blockDim.x)
    b[g] = (float)a[g];
}

}  // namespace

int sps_launch_far(sps_ctx* ctx, int op, const double* sig, double* out, bool fp32) {
  const long long NP = ctx->NP;
  const int P = ctx->T.P, N = ctx->N;
  const int ph = (op == SPS_OP_S) ? SPS_PH_FAR_S : SPS_PH_FAR_K;
  if (!fp32) {
    SpsPhase timer(ctx, ph);
    const int blocks = (int)((NP + kT64 - 1) / kT64);
    if (op == SPS_OP_S)
      k_far64<SPS_OP_S><<<blocks, kT64, 0, ctx->stream>>>(N, P, ctx->d_X, ctx->d_Nrm, ctx->d_W, sig,
                                                          ctx->d_near_ptr, ctx->d_near_idx, out);
    else
      k_far64<SPS_OP_K><<<blocks, kT64, 0, ctx->stream>>>(N, P, ctx->d_X, ctx->d_Nrm, ctx->d_W, sig,
                                                          ctx->d_near_ptr, ctx->d_near_idx, out);
    SPS_LAUNCHED(ctx);
    return SPS_OK;
  }
  const long long n3 = 3 * NP;
  {
  SpsPhase timer(ctx, SPS_PH_FAR_AUX);
  k_to_f32<<<(int)std::min<long long>((n3 + 255) / 256, 4096), 256, 0, ctx->stream>>>(n3, sig,
                                                                                     ctx->d_sig32);
  SPS_LAUNCHED(ctx);
  }
  const int bx = (int)((NP + kT32 * kTPT - 1) / (kT32 * kTPT));
  // Source splits chosen so that the grid fills whole waves of resident blocks
  // (every block does the same work, so a partial last wave idles SMs).
  static int resident = 0;
  if (!resident) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_far32<SPS_OP_K>, kT32, 0);
    resident = std::max(1, per_sm) * std::max(1, sms);
  }
  int splits = 1;
  double best = 0.0;
  for (int s = 1; s <= 32; ++s) {
    long long per_s = (NP + s - 1) / s;
    per_s = ((per_s + kTS32 - 1) / kTS32) * kTS32;
    const int s_eff = (int)((NP + per_s - 1) / per_s);
    const long long blocks = (long long)bx * s_eff;
    const long long waves = (blocks + resident - 1) / resident;
    const double eff = (double)blocks / (double)(waves * resident);
    // prefer fewer splits unless a larger count fills the machine clearly better
    if (eff > best + 0.02) {
      best = eff;
      splits = s_eff;
    }
    if (blocks >= 4LL * resident) break;
  }
  long long per = (NP + splits - 1) / splits;
  per = ((per + kTS32 - 1) / kTS32) * kTS32;
  splits = (int)((NP + per - 1) / per);
  SPS_TRY(sps_grow(ctx, &ctx->d_part, ctx->cap_part, (size_t)splits * n3));
  dim3 grid(bx, splits);
  {
  SpsPhase timer(ctx, ph);
  if (op == SPS_OP_S)
    k_far32<SPS_OP_S><<<grid, kT32, 0, ctx->stream>>>(N, P, per, ctx->d_X32, ctx->d_N32, ctx->d_W32,
                                                      ctx->d_sig32, ctx->d_near_ptr,
                                                      ctx->d_near_idx, ctx->d_part);
  else
    k_far32<SPS_OP_K><<<grid, kT32, 0, ctx->stream>>>(N, P, per, ctx->d_X32, ctx->d_N32, ctx->d_W32,
                                                      ctx->d_sig32, ctx->d_near_ptr,
                                                      ctx->d_near_idx, ctx->d_part);
  SPS_LAUNCHED(ctx);
  }
  SpsPhase timer(ctx, SPS_PH_FAR_AUX);
  const double s = (op == SPS_OP_S) ? 1.0 / (8.0 * SPS_PI) : -3.0 / (4.0 * SPS_PI);
  k_reduce_parts<<<(int)std::min<long long>((n3 + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      n3, splits, ctx->d_part, s, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}
