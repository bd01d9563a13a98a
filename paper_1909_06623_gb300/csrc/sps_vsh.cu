// Spectral (VSH) parts of the layer operators (Sec. 4.2, 5.4).
//
//  analysis   coef_s = A sigma_s: the multipliers of V, W, X in eq. rhoshexp for
//             every sphere, one small dense product per sphere (batched).
//  self       S_self = a_s Synth diag(multS) coef_s (eq. ssgext at r = 1);
//             K_self = Synth diag(multK) coef_s, the on-surface principal value
//             (exterior traction at r -> 1+ plus half the band-limited density).
//  near       for every near pair (target sphere i, source sphere j): the exterior
//             single layer of sphere j (eq. ssgshexp / ssgext) evaluated at the
//             nodes of sphere i, its velocity (S) or its traction
//             (-p I + grad u + grad u^T) n(x) (K, Sec. 4.2).
//
// Near field.  On the unit sphere the exterior field of eq. ssgext is, in
// Cartesian form (Lamb's representation with decaying solid harmonics
// phi_nm = r^{-(n+1)} Y_n^m),
//    u = grad Phi_a + x x grad Phi_d + r^2 grad Phi_alpha + x Phi_beta,
//    p = Phi_P,  Phi_* = sum_nm c*_nm phi_nm,
// with a = n sV/((2n+1)(2n+3)) + n sW/(2(2n+1)), d = sX/(2n+1),
// alpha = (2-n) sW/(2(2n-1)), beta = (n+1) sW/(2n-1), P = n sW, where
// sV, sW, sX are the expansion multipliers of the density.  This reproduces
// eq. ssgext's f^X, f^W and g exactly and f^V with the rho^W factor n/(4n+2)
// (the value that satisfies the Stokes equations; the paper prints (n+1)/(4n+2)).
// phi_nm = kappa_nm H_n^m with H_n^m = (d_x + i d_y)^m d_z^{n-m} (1/r), which obey
//    d_z H_n^m = H_{n+1}^m,  (d_x + i d_y) H_n^m = H_{n+1}^{m+1},
//    (d_x - i d_y) H_n^m = -H_{n+1}^{m-1},   H_n^{-m} = (-1)^m conj(H_n^m),
// so every derivative of a potential is again a sum over H with shifted
// coefficients, precomputed per source sphere ("fields").  Per target only the
// recurrences
//    H_m^m = -(2m-1) (x + i y) H_{m-1}^{m-1} / r^2,
//    H_{n+1}^m = -((2n+1) z H_n^m + (n^2 - m^2) H_{n-1}^m) / r^2
// and one complex multiply-add per field and (n, m >= 0) remain; nothing is
// singular at the poles.  The traction needs only the symmetric part of
// grad u, whose grad Phi_d term cancels, leaving 25 fields (6+6 Hessian
// components of Phi_a, Phi_d; grad and Hessian of Phi_alpha; grad Phi_beta;
// 2 Phi_beta - Phi_P); the velocity needs 10.
#include <type_traits>

#include "sps_dw.cuh"
#include "sps_internal.cuh"

// mixed path: VSH analysis / self synthesis on the tensor cores (BF16 split
// into three terms, FP32 accumulation) instead of FP32 CUDA-core products
#ifndef SPS_SHT_TC
#define SPS_SHT_TC 1
#endif
// 1: the source-major near field in two kernels (FP32 items at 3 CTAs per SM;
// close items in double-float), 0: one kernel doing both.  Measured on 1,000
// spheres: 0.35 ms per traction application either way.
#ifndef SPS_NEAR_SPLIT
#define SPS_NEAR_SPLIT 0
#endif

namespace {

// Batched small products out(s, r) = sum_c M[r][c] in(s, c), one sphere s per
// row of a GEMM [N x C] x [C x R]: 32 spheres x 32 rows per block, the inner
// dimension staged through shared memory in chunks of 32.
//   MODE_ANALYSIS: in = density planes (c = comp*P + node), out = coef rows.
//   MODE_SYNTH:    in = coef rows (c = VSH row), out = field planes,
//                  times a_s if scale_by_radius, plus sig/2 if half.
enum { MODE_ANALYSIS = 0, MODE_SYNTH = 1 };
constexpr int kTB = 32;

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_batched(int N, int P, int R, int C, const T* __restrict__ M,
                                                 const double* __restrict__ in,
                                                 double* __restrict__ out,
                                                 const double* __restrict__ rad,
                                                 int scale_by_radius,
                                                 const double* __restrict__ sig, int half) {
  __shared__ T sIn[kTB][kTB + 1];
  __shared__ T sM[kTB][kTB + 1];
  const long long NP = (long long)N * P;
  const int s0 = blockIdx.x * kTB, r0 = blockIdx.y * kTB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
  for (int c0 = 0; c0 < C; c0 += kTB) {
    for (int e = threadIdx.x; e < kTB * kTB; e += 256) {
      const int a = e / kTB, b = e - a * kTB;
      const int s = s0 + a, c = c0 + b, r = r0 + a;
      T v = T(0);
      if (s < N && c < C) {
        if (MODE == MODE_ANALYSIS) {
          const int comp = c / P, k = c - comp * P;
          v = (T)in[comp * NP + (long long)s * P + k];
        } else {
          v = (T)in[(long long)s * C + c];
        }
      }
      sIn[a][b] = v;
      sM[a][b] = (r < R && c < C) ? M[(long long)r * C + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int b = 0; b < kTB; ++b) {
      const T i0 = sIn[2 * ty][b], i1 = sIn[2 * ty + 1][b];
      const T m0 = sM[2 * tx][b], m1 = sM[2 * tx + 1][b];
      acc[0][0] = fma(i0, m0, acc[0][0]);
      acc[0][1] = fma(i0, m1, acc[0][1]);
      acc[1][0] = fma(i1, m0, acc[1][0]);
      acc[1][1] = fma(i1, m1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int s = s0 + 2 * ty + u, r = r0 + 2 * tx + v;
      if (s >= N || r >= R) continue;
      if (MODE == MODE_ANALYSIS) {
        double val = (double)acc[u][v];
        if (scale_by_radius) val *= rad[s];
        out[(long long)s * R + r] = val;
      } else {
        const int comp = r / P, k = r - comp * P;
        const long long idx = comp * NP + (long long)s * P + k;
        double val = (double)acc[u][v];
        if (scale_by_radius) val *= rad[s];
        if (half) val += 0.5 * sig[idx];
        out[idx] = val;
      }
    }
}

// ---------------------------------------------------------------------------
// near-field coefficient builder
// ---------------------------------------------------------------------------
enum Pot { POT_A = 0, POT_D = 1, POT_AL = 2, POT_BE = 3, POT_Q = 4 };
enum Der { D1 = 0, DX, DY, DZ, DXX, DXY, DXZ, DYY, DYZ, DZZ };

struct Field {
  unsigned char pot, der;
};

__constant__ Field c_fieldsK[sps::kFieldsK] = {
    {POT_A, DXX},  {POT_A, DXY},  {POT_A, DXZ},  {POT_A, DYY},  {POT_A, DYZ},
    {POT_A, DZZ},  {POT_D, DXX},  {POT_D, DXY},  {POT_D, DXZ},  {POT_D, DYY},
    {POT_D, DYZ},  {POT_D, DZZ},  {POT_AL, DX},  {POT_AL, DY},  {POT_AL, DZ},
    {POT_AL, DXX}, {POT_AL, DXY}, {POT_AL, DXZ}, {POT_AL, DYY}, {POT_AL, DYZ},
    {POT_AL, DZZ}, {POT_BE, DX},  {POT_BE, DY},  {POT_BE, DZ},  {POT_Q, D1}};
__constant__ Field c_fieldsS[sps::kFieldsS] = {
    {POT_A, DX},  {POT_A, DY},  {POT_A, DZ},  {POT_D, DX},  {POT_D, DY},
    {POT_D, DZ},  {POT_AL, DX}, {POT_AL, DY}, {POT_AL, DZ}, {POT_BE, D1}};

// potential coefficient c_pot(n, m) for signed m (zero outside 0 <= |m| <= n <= p).
// fac[n*6 + pot] holds the per-degree factor of each potential (host table);
// the potential a also takes fac[n*6 + 5] times sV.
__device__ double2 pot_coef(const double* __restrict__ cs, const double* __restrict__ kappa,
                            const double* __restrict__ fac, int p, int NC, int pot, int n, int m) {
  if (n < 0 || n > p || m > n || -m > n) return make_double2(0.0, 0.0);
  const int mm = m < 0 ? -m : m;
  const int ci = n * (n + 1) / 2 + mm;
  const double f = fac[n * 6 + pot];
  double re, im;
  if (pot == POT_A) {
    const double fv = fac[n * 6 + 5];
    re = fv * cs[(0 * NC + ci) * 2] + f * cs[(1 * NC + ci) * 2];
    im = fv * cs[(0 * NC + ci) * 2 + 1] + f * cs[(1 * NC + ci) * 2 + 1];
  } else if (pot == POT_D) {
    re = f * cs[(2 * NC + ci) * 2];
    im = f * cs[(2 * NC + ci) * 2 + 1];
  } else {
    re = f * cs[(1 * NC + ci) * 2];
    im = f * cs[(1 * NC + ci) * 2 + 1];
  }
  const double k = kappa[ci];
  re *= k;
  im *= k;
  if (m < 0) {  // c_{n,-m} = (-1)^m conj(c_{n,m})
    const double sg = (mm & 1) ? -1.0 : 1.0;
    re = sg * re;
    im = -sg * im;
  }
  return make_double2(re, im);
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b, double sa, double sb) {
  return make_double2(sa * a.x + sb * b.x, sa * a.y + sb * b.y);
}
__device__ __forceinline__ double2 mul_i(double2 a, double s) {  // s * i * a
  return make_double2(-s * a.y, s * a.x);
}

__device__ double2 field_coef(const double* cs, const double* kappa, const double* fac, int p, int NC,
                              Field f, int n, int m) {
  const int pot = f.pot;
  auto c = [&](int nn, int mm) { return pot_coef(cs, kappa, fac, p, NC, pot, nn, mm); };
  switch (f.der) {
    case D1: return c(n, m);
    case DX: return cadd(c(n - 1, m - 1), c(n - 1, m + 1), 0.5, -0.5);
    case DY: return mul_i(cadd(c(n - 1, m - 1), c(n - 1, m + 1), 1.0, 1.0), -0.5);
    case DZ: return c(n - 1, m);
    case DXX: {
      double2 a = cadd(c(n - 2, m - 2), c(n - 2, m + 2), 0.25, 0.25);
      return cadd(a, c(n - 2, m), 1.0, -0.5);
    }
    case DYY: {
      double2 a = cadd(c(n - 2, m - 2), c(n - 2, m + 2), -0.25, -0.25);
      return cadd(a, c(n - 2, m), 1.0, -0.5);
    }
    case DXY: return mul_i(cadd(c(n - 2, m - 2), c(n - 2, m + 2), -0.25, 0.25), 1.0);
    case DXZ: return cadd(c(n - 2, m - 1), c(n - 2, m + 1), 0.5, -0.5);
    case DYZ: return mul_i(cadd(c(n - 2, m - 1), c(n - 2, m + 1), 1.0, 1.0), -0.5);
    default: return c(n - 2, m);  // DZZ
  }
}

// fcoef[s][e][f] (complex), entries e in m'-major order, n' = m'..L
template <int F>
__global__ void k_near_coef(int N, int p, int NC, int NR, int L, int E,
                            const double* __restrict__ coef, const double* __restrict__ kappa,
                            const double* __restrict__ fac, double* __restrict__ fcoef) {
  const int s = blockIdx.x;
  const double* cs = coef + (long long)s * NR;
  const Field* fl = (F == sps::kFieldsK) ? c_fieldsK : c_fieldsS;
  for (int q = threadIdx.x; q < E * F; q += blockDim.x) {
    const int e = q / F, f = q - e * F;
    // decode entry e -> (m', n')
    int m = 0, off = 0;
    while (off + (L + 1 - m) <= e) {
      off += L + 1 - m;
      ++m;
    }
    const int n = m + (e - off);
    double2 v = field_coef(cs, kappa, fac, p, NC, fl[f], n, m);
    const double eps = (m == 0) ? 1.0 : 2.0;
    fcoef[((long long)s * E + e) * F * 2 + 2 * f] = eps * v.x;
    fcoef[((long long)s * E + e) * F * 2 + 2 * f + 1] = eps * v.y;
  }
}

using namespace sps_dw;

// 1 / sqrt(a) for the near-field expansion's arithmetic types
template <typename T>
__device__ __forceinline__ T inv_sqrt(T a) {
  return T(1) / sqrt(a);
}
template <>
__device__ __forceinline__ dw inv_sqrt<dw>(dw a) {
  return dw_rsqrt(a);
}

// ---------------------------------------------------------------------------
// near-field evaluation: one block per target sphere, one thread per node
// ---------------------------------------------------------------------------
// Contribution of source sphere j's exterior single layer at one target:
// the velocity (F = kFieldsS; times a_j by the caller) or the traction with
// target normal v (F = kFieldsK).  (x, y, z): target in sphere j's unit frame.
// cf: field coefficients of sphere j, E entries x F complex (entry-major).
// FP32 coefficients (C = float) are read as field pairs (re, re', -im, -im'),
// the entry stride padded to an even number of fields; double-float ones
// (T = dw, C = float4) as one (re hi, re lo, im hi, im lo) per field.
template <int F, typename T, typename C>
__device__ __forceinline__ void near_contrib(const C* __restrict__ cf0, int L, T x, T y, T z, T vx,
                                             T vy, T vz, T& ox, T& oy, T& oz) {
  const T r2 = x * x + y * y + z * z, ir2 = T(1) / r2;
  T acc[F];
#pragma unroll
  for (int f = 0; f < F; ++f) acc[f] = T(0);
  constexpr int FH = (F + 1) / 2;   // field pairs (FP32 path)
  float2 acc2[FH];
#pragma unroll
  for (int f = 0; f < FH; ++f) acc2[f] = make_float2(0.f, 0.f);
  T dre = inv_sqrt(r2), dim = T(0);  // H_m^m
  int e = 0;
  for (int m = 0; m <= L; ++m) {
    if (m > 0) {
      const T fm = -(T)(2 * m - 1) * ir2;
      const T re = fm * (x * dre - y * dim), im = fm * (x * dim + y * dre);
      dre = re;
      dim = im;
    }
    T hre = dre, him = dim, pre = T(0), pim = T(0);
    for (int n = m; n <= L; ++n, ++e) {
      if constexpr (std::is_same<T, dw>::value) {
        const float4* cf4 = reinterpret_cast<const float4*>(cf0) + e * F;
#pragma unroll
        for (int f = 0; f < F; ++f) {
          const float4 v = cf4[f];
          dw_mac(acc[f], dw(v.x, v.y), hre);
          dw_mac(acc[f], dw(-v.z, -v.w), him);
        }
      } else if constexpr (sizeof(C) == 4) {
        // FP32 coefficients staged per field pair as (re_f, re_f+1, -im_f,
        // -im_f+1) (zero pad for odd F): one 16-byte shared-memory load and
        // two packed FP32x2 FMAs per two fields
        const float4* cf4 = reinterpret_cast<const float4*>(cf0) + e * FH;
        const float2 hr2 = make_float2(hre, hre), hi2 = make_float2(him, him);
#pragma unroll
        for (int f2 = 0; f2 < FH; ++f2) {
          const float4 v = cf4[f2];
          acc2[f2] = __ffma2_rn(make_float2(v.x, v.y), hr2, __ffma2_rn(make_float2(v.z, v.w), hi2, acc2[f2]));
        }
      } else {
        const C* cf = cf0 + e * F * 2;
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f] = fma((T)cf[2 * f], hre, fma(-(T)cf[2 * f + 1], him, acc[f]));
      }
      const T f1 = (T)(2 * n + 1) * z, f2 = (T)(n * n - m * m);
      const T nre = -(f1 * hre + f2 * pre) * ir2, nim = -(f1 * him + f2 * pim) * ir2;
      pre = hre;
      pim = him;
      hre = nre;
      him = nim;
    }
  }
  if constexpr (std::is_same<T, dw>::value) {
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = two_sum(acc[f].h, acc[f].l);
  } else if constexpr (sizeof(C) == 4) {
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = (f & 1) ? acc2[f / 2].y : acc2[f / 2].x;
  }
  if constexpr (F == sps::kFieldsK) {
    // Hessians: [xx, xy, xz, yy, yz, zz]
    const T* HA = acc;
    const T* HD = acc + 6;
    const T* GL = acc + 12;
    const T* HL = acc + 15;
    const T* GB = acc + 21;
    const T Qs = acc[24];
    auto hv = [](const T* H, T a, T b, T c, T& o0, T& o1, T& o2) {
      o0 = H[0] * a + H[1] * b + H[2] * c;
      o1 = H[1] * a + H[3] * b + H[4] * c;
      o2 = H[2] * a + H[4] * b + H[5] * c;
    };
    T t0, t1, t2, u0, u1, u2;
    // Q v + 2 HA v
    hv(HA, vx, vy, vz, t0, t1, t2);
    T tx = Qs * vx + 2 * t0, ty = Qs * vy + 2 * t1, tz = Qs * vz + 2 * t2;
    // x x (HD v) + HD (v x x)
    hv(HD, vx, vy, vz, u0, u1, u2);
    tx += y * u2 - z * u1;
    ty += z * u0 - x * u2;
    tz += x * u1 - y * u0;
    const T cx = vy * z - vz * y, cy = vz * x - vx * z, cz = vx * y - vy * x;
    hv(HD, cx, cy, cz, u0, u1, u2);
    tx += u0;
    ty += u1;
    tz += u2;
    // 2 (GL (x.v) + x (GL.v)) + 2 r^2 HL v + x (GB.v) + GB (x.v)
    const T xv = x * vx + y * vy + z * vz;
    const T glv = GL[0] * vx + GL[1] * vy + GL[2] * vz;
    const T gbv = GB[0] * vx + GB[1] * vy + GB[2] * vz;
    hv(HL, vx, vy, vz, u0, u1, u2);
    ox = tx + 2 * (GL[0] * xv + x * glv) + 2 * r2 * u0 + x * gbv + GB[0] * xv;
    oy = ty + 2 * (GL[1] * xv + y * glv) + 2 * r2 * u1 + y * gbv + GB[1] * xv;
    oz = tz + 2 * (GL[2] * xv + z * glv) + 2 * r2 * u2 + z * gbv + GB[2] * xv;
  } else {
    const T* GA = acc;
    const T* GD = acc + 3;
    const T* GL = acc + 6;
    const T Be = acc[9];
    ox = GA[0] + (y * GD[2] - z * GD[1]) + r2 * GL[0] + x * Be;
    oy = GA[1] + (z * GD[0] - x * GD[2]) + r2 * GL[1] + y * Be;
    oz = GA[2] + (x * GD[1] - y * GD[0]) + r2 * GL[2] + z * Be;
  }
}

// One block per target sphere, one thread per node; source spheres from the
// near list staged in shared memory.  skip_r2 > 0: entries with r^2 < skip_r2
// (in units of the source radius) are left to k_near_close (FP64).
// rot (optional, N x 9): the source sphere's grid rotation Q_j; the target and
// its normal are taken into that sphere's frame (Q_j^T) and the field back
// out of it (Q_j).
template <int F, typename T>
__global__ void k_near_eval(int N, int P, int L, int E, const double* __restrict__ pos,
                            const double* __restrict__ rad, const double* __restrict__ X,
                            const double* __restrict__ Nr, const int* __restrict__ near_ptr,
                            const int* __restrict__ near_idx, const double* __restrict__ fcoef,
                            double skip_r2, const double* __restrict__ rot, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char sraw[];
  T* sc = reinterpret_cast<T*>(sraw);
  const int i = blockIdx.x;
  const long long NP = (long long)N * P;
  const int k = threadIdx.x;
  const bool valid = k < P;
  const long long g = (long long)i * P + (valid ? k : 0);
  const double gx = X[g], gy = X[NP + g], gz = X[2 * NP + g];
  T vx = 0, vy = 0, vz = 0;
  if (F == sps::kFieldsK) {
    vx = (T)Nr[g];
    vy = (T)Nr[NP + g];
    vz = (T)Nr[2 * NP + g];
  }
  double ox = 0, oy = 0, oz = 0;
  for (int q = near_ptr[i]; q < near_ptr[i + 1]; ++q) {
    const int j = near_idx[q];
    __syncthreads();
    const double* src = fcoef + (long long)j * E * F * 2;
    for (int e = threadIdx.x; e < E * F * 2; e += blockDim.x) sc[e] = (T)src[e];
    __syncthreads();
    const double aj = rad[j], ia = 1.0 / aj;
    if (skip_r2 > 0.0 && sps_close_r2(pos, ia, gx, gy, gz, j) < skip_r2) continue;
    T x = (T)((gx - pos[3 * j]) * ia), y = (T)((gy - pos[3 * j + 1]) * ia),
      z = (T)((gz - pos[3 * j + 2]) * ia);
    T wx = vx, wy = vy, wz = vz;
    const double* Q = rot ? rot + 9 * j : nullptr;
    if (Q) {
      sps_rot_t(Q, x, y, z);
      if (F == sps::kFieldsK) sps_rot_t(Q, wx, wy, wz);
    }
    T tx, ty, tz;
    near_contrib<F, T, T>(sc, L, x, y, z, wx, wy, wz, tx, ty, tz);
    if (Q) sps_rot_n(Q, tx, ty, tz);
    if (F == sps::kFieldsK) {
      ox += (double)tx;
      oy += (double)ty;
      oz += (double)tz;
    } else {
      ox += aj * (double)tx;
      oy += aj * (double)ty;
      oz += aj * (double)tz;
    }
  }
  if (valid) {
    out[g] += ox;
    out[NP + g] += oy;
    out[2 * NP + g] += oz;
  }
}

// Mixed-precision near field: k_near_eval with FP32 field coefficients
// (staged as float2), the target's position in the source frame formed in
// FP32 from per-source values computed once per block, and compensated FP32
// sums per target.  Entries closer than kCloseRadius source radii belong to
// k_near_close: the FP32 distance decides where it is clear by a wide
// margin, the close list's own FP64 test inside the margin, so the two
// kernels split the entries exactly as the list does.
template <int F>
__global__ void k_near_eval32(int N, int P, int L, int E, const double* __restrict__ pos,
                              const double* __restrict__ rad, const double* __restrict__ X,
                              const double* __restrict__ Nr, const int* __restrict__ near_ptr,
                              const int* __restrict__ near_idx, const float* __restrict__ fcoef,
                              const double* __restrict__ rot, double* __restrict__ out) {
  constexpr int FP = (F + 1) & ~1;   // padded field count of a staged entry
  __shared__ float s_rot[9];   // Q_j of the staged source (oriented grids)
  extern __shared__ __align__(16) unsigned char sraw[];
  float2* sc2 = reinterpret_cast<float2*>(sraw);
  __shared__ float s_geo[5];   // (c_i - c_j) / a_j, 1 / a_j, a_j
  __shared__ double s_iad;     // 1 / a_j in FP64
  const int i = blockIdx.x;
  const long long NP = (long long)N * P;
  const int k = threadIdx.x;
  const bool valid = k < P;
  const long long g = (long long)i * P + (valid ? k : 0);
  const double ci0 = pos[3 * i], ci1 = pos[3 * i + 1], ci2 = pos[3 * i + 2];
  const float lx = (float)(X[g] - ci0), ly = (float)(X[NP + g] - ci1), lz = (float)(X[2 * NP + g] - ci2);
  float vx = 0.f, vy = 0.f, vz = 0.f;
  if (F == sps::kFieldsK) {
    vx = (float)Nr[g];
    vy = (float)Nr[NP + g];
    vz = (float)Nr[2 * NP + g];
  }
  const double lim = sps::kCloseRadius * sps::kCloseRadius;
  const float lo = (float)(lim * (1.0 - 1e-4)), hi = (float)(lim * (1.0 + 1e-4));
  float ox = 0.f, oy = 0.f, oz = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;   // sums, compensations
  auto kadd = [](float& sum, float& c, float v) {
    const float y = v - c, t = sum + y;
    c = (t - sum) - y;
    sum = t;
  };
  for (int q = near_ptr[i]; q < near_ptr[i + 1]; ++q) {
    const int j = near_idx[q];
    __syncthreads();
    const float2* src = reinterpret_cast<const float2*>(fcoef + (long long)j * E * F * 2);
    // field pairs of entry e: (re_2k, re_2k+1, -im_2k, -im_2k+1), one warp per entry
    {
      float4* sc4 = reinterpret_cast<float4*>(sc2);
      const int lane = threadIdx.x & 31;
      for (int e = threadIdx.x >> 5; e < E; e += blockDim.x >> 5)
        if (lane < FP / 2) {
          const float2 a = src[e * F + 2 * lane];
          const float2 b = (2 * lane + 1 < F) ? src[e * F + 2 * lane + 1] : make_float2(0.f, 0.f);
          sc4[e * (FP / 2) + lane] = make_float4(a.x, b.x, -a.y, -b.y);
        }
    }
    if (threadIdx.x == 0) {
      const double aj = rad[j], ia = 1.0 / aj;
      s_geo[0] = (float)((ci0 - pos[3 * j]) * ia);
      s_geo[1] = (float)((ci1 - pos[3 * j + 1]) * ia);
      s_geo[2] = (float)((ci2 - pos[3 * j + 2]) * ia);
      s_geo[3] = (float)ia;
      s_geo[4] = (float)aj;
      s_iad = ia;
      if (rot)
        for (int c = 0; c < 9; ++c) s_rot[c] = (float)rot[9 * j + c];
    }
    __syncthreads();
    const float ia = s_geo[3];
    const float x = fmaf(lx, ia, s_geo[0]), y = fmaf(ly, ia, s_geo[1]), z = fmaf(lz, ia, s_geo[2]);
    const float r2 = x * x + y * y + z * z;
    if (r2 < hi) {
      if (r2 < lo) continue;
      if (sps_close_r2(pos, s_iad, X[g], X[NP + g], X[2 * NP + g], j) < lim) continue;
    }
    float xr = x, yr = y, zr = z, wx = vx, wy = vy, wz = vz;
    if (rot) {
      sps_rot_t(s_rot, xr, yr, zr);
      if (F == sps::kFieldsK) sps_rot_t(s_rot, wx, wy, wz);
    }
    float tx, ty, tz;
    near_contrib<F, float, float>(reinterpret_cast<const float*>(sc2), L, xr, yr, zr, wx, wy, wz, tx, ty, tz);
    if (rot) sps_rot_n(s_rot, tx, ty, tz);
    if (F == sps::kFieldsS) {
      const float aj = s_geo[4];
      tx *= aj;
      ty *= aj;
      tz *= aj;
    }
    kadd(ox, ex, tx);
    kadd(oy, ey, ty);
    kadd(oz, ez, tz);
  }
  if (valid) {
    out[g] += (double)ox - (double)ex;
    out[NP + g] += (double)oy - (double)ey;
    out[2 * NP + g] += (double)oz - (double)ez;
  }
}

// FP64 near entries of the mixed path: one thread per close node, its close
// source spheres in near-list order (coefficients read through the cache).
template <int F>
__global__ void k_near_close(int N, int P, int L, int E, int n_close, const int* __restrict__ cnode,
                             const int* __restrict__ cptr, const int* __restrict__ csrc,
                             const double* __restrict__ pos, const double* __restrict__ rad,
                             const double* __restrict__ X, const double* __restrict__ Nr,
                             const double* __restrict__ fcoef, const double* __restrict__ rot,
                             double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_close) return;
  const long long NP = (long long)N * P;
  const long long g = cnode[t];
  const double gx = X[g], gy = X[NP + g], gz = X[2 * NP + g];
  double vx = 0, vy = 0, vz = 0;
  if (F == sps::kFieldsK) {
    vx = Nr[g];
    vy = Nr[NP + g];
    vz = Nr[2 * NP + g];
  }
  double ox = 0, oy = 0, oz = 0;
  for (int q = cptr[t]; q < cptr[t + 1]; ++q) {
    const int j = csrc[q];
    const double aj = rad[j], ia = 1.0 / aj;
    double x = (gx - pos[3 * j]) * ia, y = (gy - pos[3 * j + 1]) * ia, z = (gz - pos[3 * j + 2]) * ia;
    double wx = vx, wy = vy, wz = vz;
    const double* Q = rot ? rot + 9 * j : nullptr;
    if (Q) {
      sps_rot_t(Q, x, y, z);
      if (F == sps::kFieldsK) sps_rot_t(Q, wx, wy, wz);
    }
    double tx, ty, tz;
    near_contrib<F, double, double>(fcoef + (long long)j * E * F * 2, L, x, y, z, wx, wy, wz, tx, ty, tz);
    if (Q) sps_rot_n(Q, tx, ty, tz);
    if (F == sps::kFieldsK) {
      ox += tx;
      oy += ty;
      oz += tz;
    } else {
      ox += aj * tx;
      oy += aj * ty;
      oz += aj * tz;
    }
  }
  out[g] += ox;
  out[NP + g] += oy;
  out[2 * NP + g] += oz;
}

template <int F, typename T>
int launch_near_eval(sps_ctx* ctx, double skip_r2, double* out) {
  const int N = ctx->N, P = ctx->T.P, L = ctx->T.L, E = ctx->T.E;
  const int threads = ((P + 31) / 32) * 32;
  const size_t sm = sizeof(T) * E * F * 2;
  if (sm > 48 * 1024)
    SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_eval<F, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm));
  k_near_eval<F, T><<<N, threads, sm, ctx->stream>>>(N, P, L, E, ctx->d_pos, ctx->d_rad, ctx->d_X,
                                                      ctx->d_Nrm, ctx->d_near_ptr, ctx->d_near_idx,
                                                      ctx->d_fcoef, skip_r2, sps_rot(ctx), out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

template <int F>
int launch_near_eval32(sps_ctx* ctx, double* out) {
  const int N = ctx->N, P = ctx->T.P, L = ctx->T.L, E = ctx->T.E;
  const int threads = ((P + 31) / 32) * 32;
  const size_t sm = sizeof(float) * E * ((F + 1) & ~1) * 2;
  if (sm > 48 * 1024)
    SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_eval32<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm));
  k_near_eval32<F><<<N, threads, sm, ctx->stream>>>(N, P, L, E, ctx->d_pos, ctx->d_rad, ctx->d_X,
                                                     ctx->d_Nrm, ctx->d_near_ptr, ctx->d_near_idx,
                                                     ctx->d_fcoef32, sps_rot(ctx), out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// The same entries in double-float arithmetic (coefficients as hi + lo FP32
// pairs): FP64 only to place the target in the source frame and to add up.
template <int F>
__global__ void k_near_close_dw(int N, int P, int L, int E, int n_close, const int* __restrict__ cnode,
                                const int* __restrict__ cptr, const int* __restrict__ csrc,
                                const double* __restrict__ pos, const double* __restrict__ rad,
                                const double* __restrict__ X, const double* __restrict__ Nr,
                                const float4* __restrict__ fcoef, const double* __restrict__ rot,
                                double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_close) return;
  const long long NP = (long long)N * P;
  const long long g = cnode[t];
  const double gx = X[g], gy = X[NP + g], gz = X[2 * NP + g];
  double nx = 0.0, ny = 0.0, nz = 0.0;
  if (F == sps::kFieldsK) {
    nx = Nr[g];
    ny = Nr[NP + g];
    nz = Nr[2 * NP + g];
  }
  dw vx = dw_of(nx), vy = dw_of(ny), vz = dw_of(nz);
  double ox = 0, oy = 0, oz = 0;
  for (int q = cptr[t]; q < cptr[t + 1]; ++q) {
    const int j = csrc[q];
    const double aj = rad[j], ia = 1.0 / aj;
    double x64 = (gx - pos[3 * j]) * ia, y64 = (gy - pos[3 * j + 1]) * ia, z64 = (gz - pos[3 * j + 2]) * ia;
    const double* Q = rot ? rot + 9 * j : nullptr;
    if (Q) {
      sps_rot_t(Q, x64, y64, z64);
      if (F == sps::kFieldsK) {
        double mx = nx, my = ny, mz = nz;
        sps_rot_t(Q, mx, my, mz);
        vx = dw_of(mx);
        vy = dw_of(my);
        vz = dw_of(mz);
      }
    }
    const dw x = dw_of(x64), y = dw_of(y64), z = dw_of(z64);
    dw tx, ty, tz;
    near_contrib<F, dw, float4>(fcoef + (long long)j * E * F, L, x, y, z, vx, vy, vz, tx, ty, tz);
    const double s = (F == sps::kFieldsK) ? 1.0 : aj;
    double rx = s * dw_val(tx), ry = s * dw_val(ty), rz = s * dw_val(tz);
    if (Q) sps_rot_n(Q, rx, ry, rz);
    ox += rx;
    oy += ry;
    oz += rz;
  }
  out[g] += ox;
  out[NP + g] += oy;
  out[2 * NP + g] += oz;
}

// ---------------------------------------------------------------------------
// Source-major near field (mixed path).  One CTA per source sphere j stages
// j's field coefficients once (FP32 pairs and double-float) and evaluates them
// at every node of every near target sphere i of j: the items (pair, node).
// The close / far split is the one of the close list (FP32 distance outside a
// 1e-4 band around kCloseRadius, the list's FP64 test inside it).  Far items
// use the FP32 expansion (k_near_eval32's arithmetic); close items are
// collected in shared memory and evaluated afterwards in double-float
// (k_near_close_dw's arithmetic), so no warp diverges on them.  Each item's
// field goes to buf at its target-major pair slot; k_near_reduce adds a
// node's pairs in near-list order in FP64 (deterministic).
// ---------------------------------------------------------------------------
constexpr int kNS = 256;
constexpr int kMaxClose = 1024;   // close items listed per CTA (beyond: a rescan of all items)

// Item it of source j (target node k of the qq-th near target): its
// position relative to the source centre in source radii (FP32, before any
// rotation) and whether it is a close item.  The split is the close list's:
// decided in FP32 outside a 1e-4 band around kCloseRadius, by the list's
// FP64 test inside it.  Returns false for a missing reverse slot (q < 0).
__device__ __forceinline__ bool near_item(int it, int j, int q0, int P, long long NP,
                                          const int* __restrict__ near_idx, const int* __restrict__ rev,
                                          const float* __restrict__ rel32, const float* __restrict__ geo,
                                          const double* __restrict__ pos, const double* __restrict__ X,
                                          float ia, double iad, float lo, float hi, double lim, long long& g,
                                          int& q, int& k, float& x, float& y, float& z, bool& close) {
  const int qq = it / P;
  k = it - qq * P;
  const int i = near_idx[q0 + qq];
  q = rev[q0 + qq];
  if (q < 0) return false;   // (cannot happen: the near relation is symmetric to the bit)
  g = (long long)i * P + k;
  x = fmaf(rel32[g], ia, geo[3 * q]);
  y = fmaf(rel32[NP + g], ia, geo[3 * q + 1]);
  z = fmaf(rel32[2 * NP + g], ia, geo[3 * q + 2]);
  const float r2 = x * x + y * y + z * z;
  close = r2 < hi && (r2 < lo || sps_close_r2(pos, iad, X[g], X[NP + g], X[2 * NP + g], j) < lim);
  return true;
}

template <int F>
__device__ __forceinline__ void near_src_close(int it, int j, int q0, int P, int L, long long NP, long long NQ,
                                               const double* __restrict__ pos, double aj, double iad,
                                               const double* __restrict__ X, const double* __restrict__ Nr,
                                               const int* __restrict__ near_idx, const int* __restrict__ rev,
                                               const float4* cdw, const double* Q, double* __restrict__ buf) {
  const int qq = it / P, k = it - qq * P;
  const int i = near_idx[q0 + qq], q = rev[q0 + qq];
  if (q < 0) return;   // (cannot happen: the near relation is symmetric to the bit)
  const long long g = (long long)i * P + k, o = (long long)q * P + k;
  double x64 = (X[g] - pos[3 * j]) * iad, y64 = (X[NP + g] - pos[3 * j + 1]) * iad,
         z64 = (X[2 * NP + g] - pos[3 * j + 2]) * iad;
  double nx = 0.0, ny = 0.0, nz = 0.0;
  if (F == sps::kFieldsK) {
    nx = Nr[g];
    ny = Nr[NP + g];
    nz = Nr[2 * NP + g];
  }
  if (Q) {
    sps_rot_t(Q, x64, y64, z64);
    if (F == sps::kFieldsK) sps_rot_t(Q, nx, ny, nz);
  }
  dw tx, ty, tz;
  near_contrib<F, dw, float4>(cdw, L, dw_of(x64), dw_of(y64), dw_of(z64), dw_of(nx), dw_of(ny), dw_of(nz), tx,
                              ty, tz);
  const double sc = (F == sps::kFieldsK) ? 1.0 : aj;
  double rx = sc * dw_val(tx), ry = sc * dw_val(ty), rz = sc * dw_val(tz);
  if (Q) sps_rot_n(Q, rx, ry, rz);
  buf[o] = rx;
  buf[NQ + o] = ry;
  buf[2 * NQ + o] = rz;
}

// FAR_ONLY = 1: the FP32 items only (close items are left to k_near_src_close,
// and the double-float path does not weigh on this kernel's registers)
template <int F, int FAR_ONLY>
__global__ void __launch_bounds__(kNS, FAR_ONLY ? 3 : 2) k_near_src(int N, int P, int L, int E, long long NQ,
                                                 const double* __restrict__ pos, const double* __restrict__ rad,
                                                 const double* __restrict__ X, const double* __restrict__ Nr,
                                                 const float* __restrict__ rel32, const float* __restrict__ N32,
                                                 const int* __restrict__ near_ptr, const int* __restrict__ near_idx,
                                                 const int* __restrict__ rev, const float* __restrict__ geo,
                                                 const float* __restrict__ fcoef32,
                                                 const float4* __restrict__ fcoefdw,
                                                 const double* __restrict__ rot, double* __restrict__ buf) {
  constexpr int FP = (F + 1) & ~1;
  extern __shared__ __align__(16) unsigned char sraw[];
  float4* c32 = reinterpret_cast<float4*>(sraw);     // E x FP/2 field pairs
  float4* cdw = c32 + E * (FP / 2);                 // E x F double-float fields (unless FAR_ONLY)
  __shared__ float s_rot[9];
  __shared__ double s_rotd[9];
  __shared__ int s_ncl;
  __shared__ int s_cl[kMaxClose];
  const int j = blockIdx.x;
  const int q0 = near_ptr[j], nn = near_ptr[j + 1] - q0;
  if (nn == 0) return;                               // uniform over the block
  const float2* src = reinterpret_cast<const float2*>(fcoef32 + (long long)j * E * F * 2);
  for (int t = threadIdx.x; t < E * (FP / 2); t += kNS) {
    const int e = t / (FP / 2), l = t - e * (FP / 2);
    const float2 a = src[e * F + 2 * l];
    const float2 b = (2 * l + 1 < F) ? src[e * F + 2 * l + 1] : make_float2(0.f, 0.f);
    c32[t] = make_float4(a.x, b.x, -a.y, -b.y);
  }
  if (threadIdx.x == 0) {
    s_ncl = 0;
    if (rot)
      for (int c = 0; c < 9; ++c) {
        s_rotd[c] = rot[9 * j + c];
        s_rot[c] = (float)rot[9 * j + c];
      }
  }
  __syncthreads();
  const long long NP = (long long)N * P;
  const double aj = rad[j], iad = 1.0 / aj;
  const float ia = (float)iad, ajf = (float)aj;
  const double lim = sps::kCloseRadius * sps::kCloseRadius;
  const float lo = (float)(lim * (1.0 - 1e-4)), hi = (float)(lim * (1.0 + 1e-4));
  const double* Qd = rot ? s_rotd : nullptr;
  const int items = nn * P;
  for (int it = threadIdx.x; it < items; it += kNS) {
    long long g;
    int q, k;
    float x, y, z;
    bool close;
    if (!near_item(it, j, q0, P, NP, near_idx, rev, rel32, geo, pos, X, ia, iad, lo, hi, lim, g, q, k, x, y, z,
                   close))
      continue;
    if (close) {
      if (FAR_ONLY) continue;
      const int c = atomicAdd(&s_ncl, 1);
      if (c < kMaxClose) s_cl[c] = it;
      continue;
    }
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (F == sps::kFieldsK) {
      vx = N32[g];
      vy = N32[NP + g];
      vz = N32[2 * NP + g];
    }
    if (rot) {
      sps_rot_t(s_rot, x, y, z);
      if (F == sps::kFieldsK) sps_rot_t(s_rot, vx, vy, vz);
    }
    float tx, ty, tz;
    near_contrib<F, float, float>(reinterpret_cast<const float*>(c32), L, x, y, z, vx, vy, vz, tx, ty, tz);
    if (rot) sps_rot_n(s_rot, tx, ty, tz);
    if (F == sps::kFieldsS) {
      tx *= ajf;
      ty *= ajf;
      tz *= ajf;
    }
    const long long o = (long long)q * P + k;
    buf[o] = tx;
    buf[NQ + o] = ty;
    buf[2 * NQ + o] = tz;
  }
  if (FAR_ONLY) return;
  // close items: the source's double-float coefficients are staged only by
  // CTAs that have some (most sources have none)
  __syncthreads();
  const int ncl = s_ncl;
  if (ncl == 0) return;                              // uniform over the block
  const float4* dsrc = fcoefdw + (long long)j * E * F;
  for (int t = threadIdx.x; t < E * F; t += kNS) cdw[t] = dsrc[t];
  __syncthreads();
  if (ncl <= kMaxClose) {
    for (int c = threadIdx.x; c < ncl; c += kNS)
      near_src_close<F>(s_cl[c], j, q0, P, L, NP, NQ, pos, aj, iad, X, Nr, near_idx, rev, cdw, Qd, buf);
    return;
  }
  // the list overflowed: find every close item again (the same test) instead
  for (int it = threadIdx.x; it < items; it += kNS) {
    long long g;
    int q, k;
    float x, y, z;
    bool close;
    if (near_item(it, j, q0, P, NP, near_idx, rev, rel32, geo, pos, X, ia, iad, lo, hi, lim, g, q, k, x, y, z,
                  close) && close)
      near_src_close<F>(it, j, q0, P, L, NP, NQ, pos, aj, iad, X, Nr, near_idx, rev, cdw, Qd, buf);
  }
}

// The close items of source j (the same split as k_near_src's), in
// double-float with j's coefficients staged once: the companion of
// k_near_src<F, 1>.
constexpr int kNC = 128;
template <int F>
__global__ void __launch_bounds__(kNC) k_near_src_close(int N, int P, int L, int E, long long NQ,
                                                        const double* __restrict__ pos,
                                                        const double* __restrict__ rad,
                                                        const double* __restrict__ X, const double* __restrict__ Nr,
                                                        const float* __restrict__ rel32,
                                                        const int* __restrict__ near_ptr,
                                                        const int* __restrict__ near_idx,
                                                        const int* __restrict__ rev, const float* __restrict__ geo,
                                                        const float4* __restrict__ fcoefdw,
                                                        const double* __restrict__ rot, double* __restrict__ buf) {
  extern __shared__ __align__(16) unsigned char sraw[];
  float4* cdw = reinterpret_cast<float4*>(sraw);    // E x F double-float fields
  __shared__ double s_rotd[9];
  __shared__ int s_ncl;
  __shared__ int s_cl[kMaxClose];
  const int j = blockIdx.x;
  const int q0 = near_ptr[j], nn = near_ptr[j + 1] - q0;
  if (nn == 0) return;
  if (threadIdx.x == 0) {
    s_ncl = 0;
    if (rot)
      for (int c = 0; c < 9; ++c) s_rotd[c] = rot[9 * j + c];
  }
  __syncthreads();
  const long long NP = (long long)N * P;
  const double aj = rad[j], iad = 1.0 / aj;
  const float ia = (float)iad;
  const double lim = sps::kCloseRadius * sps::kCloseRadius;
  const float lo = (float)(lim * (1.0 - 1e-4)), hi = (float)(lim * (1.0 + 1e-4));
  const double* Qd = rot ? s_rotd : nullptr;
  const int items = nn * P;
  for (int it = threadIdx.x; it < items; it += kNC) {
    const int qq = it / P, k = it - qq * P;
    const int i = near_idx[q0 + qq];
    const int q = rev[q0 + qq];
    if (q < 0) continue;
    const long long g = (long long)i * P + k;
    const float x = fmaf(rel32[g], ia, geo[3 * q]), y = fmaf(rel32[NP + g], ia, geo[3 * q + 1]),
                z = fmaf(rel32[2 * NP + g], ia, geo[3 * q + 2]);
    const float r2 = x * x + y * y + z * z;
    if (r2 < hi && (r2 < lo || sps_close_r2(pos, iad, X[g], X[NP + g], X[2 * NP + g], j) < lim)) {
      const int c = atomicAdd(&s_ncl, 1);
      if (c < kMaxClose) s_cl[c] = it;
    }
  }
  __syncthreads();
  const int ncl = s_ncl;
  if (ncl == 0) return;
  const float4* dsrc = fcoefdw + (long long)j * E * F;
  for (int t = threadIdx.x; t < E * F; t += kNC) cdw[t] = dsrc[t];
  __syncthreads();
  for (int c = threadIdx.x; c < min(ncl, kMaxClose); c += kNC)
    near_src_close<F>(s_cl[c], j, q0, P, L, NP, NQ, pos, aj, iad, X, Nr, near_idx, rev, cdw, Qd, buf);
  // more close items than the list holds: every close item is found again and
  // evaluated in place (the writes are idempotent, so the listed ones may repeat)
  if (ncl > kMaxClose) {
    for (int it = threadIdx.x; it < items; it += kNC) {
      const int qq = it / P, k = it - qq * P;
      const int i = near_idx[q0 + qq];
      const int q = rev[q0 + qq];
      if (q < 0) continue;
      const long long g = (long long)i * P + k;
      const float x = fmaf(rel32[g], ia, geo[3 * q]), y = fmaf(rel32[NP + g], ia, geo[3 * q + 1]),
                  z = fmaf(rel32[2 * NP + g], ia, geo[3 * q + 2]);
      const float r2 = x * x + y * y + z * z;
      if (r2 < hi && (r2 < lo || sps_close_r2(pos, iad, X[g], X[NP + g], X[2 * NP + g], j) < lim))
        near_src_close<F>(it, j, q0, P, L, NP, NQ, pos, aj, iad, X, Nr, near_idx, rev, cdw, Qd, buf);
    }
  }
}

// out[g] += sum over the near pairs q of g's sphere (near-list order) of buf
__global__ void k_near_reduce(int N, int P, long long NQ, const int* __restrict__ near_ptr,
                              const double* __restrict__ buf, double* __restrict__ out) {
  const long long NP = (long long)N * P;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NP;
       g += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(g / P), k = (int)(g - (long long)i * P);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int q = near_ptr[i]; q < near_ptr[i + 1]; ++q) {
      const long long o = (long long)q * P + k;
      sx += buf[o];
      sy += buf[NQ + o];
      sz += buf[2 * NQ + o];
    }
    out[g] += sx;
    out[NP + g] += sy;
    out[2 * NP + g] += sz;
  }
}

template <int F>
int launch_near_src(sps_ctx* ctx, double* out) {
  const int N = ctx->N, P = ctx->T.P, L = ctx->T.L, E = ctx->T.E;
  const long long NQ = (long long)ctx->n_near * P;
  SPS_TRY(sps_grow(ctx, &ctx->d_near_buf, ctx->cap_near_buf, 3 * (size_t)NQ));
  constexpr int FP = (F + 1) & ~1;
  const float4* fdw = reinterpret_cast<const float4*>(ctx->d_fcoefdw);
  if (SPS_NEAR_SPLIT) {
    // FP32 items, then the close items of each source in double-float
    const size_t sm = sizeof(float4) * (size_t)E * (FP / 2);
    if (sm > 48 * 1024)
      SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_src<F, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_near_src<F, 1><<<N, kNS, sm, ctx->stream>>>(N, P, L, E, NQ, ctx->d_pos, ctx->d_rad, ctx->d_X, ctx->d_Nrm,
                                                  ctx->d_rel32, ctx->d_N32, ctx->d_near_ptr, ctx->d_near_idx,
                                                  ctx->d_near_rev, ctx->d_near_geo, ctx->d_fcoef32, fdw,
                                                  sps_rot(ctx), ctx->d_near_buf);
    SPS_LAUNCHED(ctx);
    const size_t smc = sizeof(float4) * (size_t)E * F;
    if (smc > 48 * 1024)
      SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_src_close<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smc));
    k_near_src_close<F><<<N, kNC, smc, ctx->stream>>>(N, P, L, E, NQ, ctx->d_pos, ctx->d_rad, ctx->d_X,
                                                      ctx->d_Nrm, ctx->d_rel32, ctx->d_near_ptr, ctx->d_near_idx,
                                                      ctx->d_near_rev, ctx->d_near_geo, fdw, sps_rot(ctx),
                                                      ctx->d_near_buf);
    SPS_LAUNCHED(ctx);
  } else {
    const size_t sm = sizeof(float4) * (size_t)E * (FP / 2 + F);
    if (sm > 48 * 1024)
      SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_src<F, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_near_src<F, 0><<<N, kNS, sm, ctx->stream>>>(N, P, L, E, NQ, ctx->d_pos, ctx->d_rad, ctx->d_X, ctx->d_Nrm,
                                                  ctx->d_rel32, ctx->d_N32, ctx->d_near_ptr, ctx->d_near_idx,
                                                  ctx->d_near_rev, ctx->d_near_geo, ctx->d_fcoef32, fdw,
                                                  sps_rot(ctx), ctx->d_near_buf);
    SPS_LAUNCHED(ctx);
  }
  const long long NP = (long long)N * P;
  k_near_reduce<<<(int)std::min<long long>((NP + 255) / 256, 8 * 152), 256, 0, ctx->stream>>>(
      N, P, NQ, ctx->d_near_ptr, ctx->d_near_buf, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

#ifndef SPS_CLOSE_DW
#define SPS_CLOSE_DW 1
#endif
// 1: the mixed path's near field runs source-major (k_near_src); 0: the
// target-major kernels k_near_eval32 + k_near_close_dw
#ifndef SPS_NEAR_SRC
#define SPS_NEAR_SRC 1
#endif
template <int F>
int launch_near_close(sps_ctx* ctx, double* out) {
  if (SPS_CLOSE_DW) {
    if (ctx->n_close == 0) return SPS_OK;
    k_near_close_dw<F><<<(ctx->n_close + 63) / 64, 64, 0, ctx->stream>>>(
        ctx->N, ctx->T.P, ctx->T.L, ctx->T.E, ctx->n_close, ctx->d_close_node, ctx->d_close_ptr,
        ctx->d_close_src, ctx->d_pos, ctx->d_rad, ctx->d_X, ctx->d_Nrm,
        reinterpret_cast<const float4*>(ctx->d_fcoefdw), sps_rot(ctx), out);
    SPS_LAUNCHED(ctx);
    return SPS_OK;
  }
  if (ctx->n_close == 0) return SPS_OK;
  k_near_close<F><<<(ctx->n_close + 63) / 64, 64, 0, ctx->stream>>>(
      ctx->N, ctx->T.P, ctx->T.L, ctx->T.E, ctx->n_close, ctx->d_close_node, ctx->d_close_ptr,
      ctx->d_close_src, ctx->d_pos, ctx->d_rad, ctx->d_X, ctx->d_Nrm, ctx->d_fcoef, sps_rot(ctx), out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// out[s][r] (+)= sum over row r of a sparse map applied to in[s][:]
// (out32: the result rounded to FP32; outdw: split into FP32 hi + lo; same
// layout)
__global__ void k_sparse_rows(int N, int rows, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ val, const double* __restrict__ in, int in_ld,
                              double* __restrict__ out, int out_ld, int accumulate,
                              float* __restrict__ out32, float2* __restrict__ outdw) {
  const long long tot = (long long)N * rows;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(q / rows), r = (int)(q - (long long)s * rows);
    const double* x = in + (long long)s * in_ld;
    double acc = 0.0;
    for (int k = rp[r]; k < rp[r + 1]; ++k) acc = fma(val[k], x[ci[k]], acc);
    double* y = out + (long long)s * out_ld + r;
    *y = accumulate ? *y + acc : acc;
    if (out32) out32[(long long)s * out_ld + r] = (float)acc;
    if (outdw) {
      const float h = __double2float_rn(acc);
      outdw[(long long)s * out_ld + r] = make_float2(h, __double2float_rn(acc - (double)h));
    }
  }
}

}  // namespace

int sps_launch_sparse_rows(sps_ctx* ctx, const sps_ctx::Sparse& m, int nsph, const double* in, int in_ld,
                           double* out, int out_ld, int accumulate, float* out32, float2* outdw) {
  const long long tot = (long long)nsph * m.rows;
  k_sparse_rows<<<(int)std::min<long long>((tot + 255) / 256, 8 * 152), 256, 0, ctx->stream>>>(
      nsph, m.rows, m.rp, m.ci, m.v, in, in_ld, out, out_ld, accumulate, accumulate ? nullptr : out32,
      accumulate ? nullptr : outdw);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// The coefficient builder is linear in the VSH coefficients with constant
// weights; run it once on unit coefficient vectors to obtain that map as a
// sparse matrix (and its transpose, for the adjoint).
template <int F>
static int field_map(sps_ctx* ctx, sps_ctx::Sparse& fm, sps_ctx::Sparse& fmt) {
  const int NR = ctx->T.NR, E = ctx->T.E, NC = ctx->T.NC, L = ctx->T.L, p = ctx->T.p;
  const int W = E * F * 2;
  std::vector<double> eye((size_t)NR * NR, 0.0), out((size_t)NR * W);
  for (int r = 0; r < NR; ++r) eye[(size_t)r * NR + r] = 1.0;
  double *d_in = nullptr, *d_out = nullptr;
  SPS_CUDA(ctx, cudaMalloc(&d_in, eye.size() * sizeof(double)));
  SPS_CUDA(ctx, cudaMalloc(&d_out, out.size() * sizeof(double)));
  SPS_CUDA(ctx, cudaMemcpy(d_in, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice));
  k_near_coef<F><<<NR, 256, 0, ctx->stream>>>(NR, p, NC, NR, L, E, d_in, ctx->d_kappa, ctx->d_potfac, d_out);
  SPS_LAUNCHED(ctx);
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  SPS_CUDA(ctx, cudaMemcpy(out.data(), d_out, out.size() * sizeof(double), cudaMemcpyDeviceToHost));
  cudaFree(d_in);
  cudaFree(d_out);
  // out[r][k] = FM[k][r]
  std::vector<int> rp(W + 1, 0), rpt(NR + 1, 0), ci, cit;
  std::vector<double> val, valt;
  for (int k = 0; k < W; ++k) {
    for (int r = 0; r < NR; ++r) {
      const double x = out[(size_t)r * W + k];
      if (x != 0.0) {
        ci.push_back(r);
        val.push_back(x);
      }
    }
    rp[k + 1] = (int)ci.size();
  }
  for (int r = 0; r < NR; ++r) {
    for (int k = 0; k < W; ++k) {
      const double x = out[(size_t)r * W + k];
      if (x != 0.0) {
        cit.push_back(k);
        valt.push_back(x);
      }
    }
    rpt[r + 1] = (int)cit.size();
  }
  auto up = [&](sps_ctx::Sparse& m, int rows, int cols, const std::vector<int>& a, const std::vector<int>& b,
                const std::vector<double>& c) -> int {
    m.rows = rows;
    m.cols = cols;
    m.nnz = (int)c.size();
    SPS_CUDA(ctx, cudaMalloc(&m.rp, sizeof(int) * a.size()));
    SPS_CUDA(ctx, cudaMalloc(&m.ci, sizeof(int) * std::max<size_t>(1, b.size())));
    SPS_CUDA(ctx, cudaMalloc(&m.v, sizeof(double) * std::max<size_t>(1, c.size())));
    SPS_CUDA(ctx, cudaMemcpy(m.rp, a.data(), sizeof(int) * a.size(), cudaMemcpyHostToDevice));
    SPS_CUDA(ctx, cudaMemcpy(m.ci, b.data(), sizeof(int) * b.size(), cudaMemcpyHostToDevice));
    SPS_CUDA(ctx, cudaMemcpy(m.v, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice));
    return SPS_OK;
  };
  SPS_TRY(up(fm, W, NR, rp, ci, val));
  SPS_TRY(up(fmt, NR, W, rpt, cit, valt));
  return SPS_OK;
}

int sps_build_field_maps(sps_ctx* ctx) {
  SPS_TRY(field_map<sps::kFieldsK>(ctx, ctx->fmK, ctx->fmKt));
  SPS_TRY(field_map<sps::kFieldsS>(ctx, ctx->fmS, ctx->fmSt));
  return SPS_OK;
}

int sps_launch_batched(sps_ctx* ctx, int mode, const double* M, int R, int C, const double* in, double* out,
                       int scale_by_radius, const double* sig, int half) {
  SpsPhase timer(ctx, SPS_PH_SELF);
  const int N = ctx->N, P = ctx->T.P;
  dim3 grid((N + kTB - 1) / kTB, (R + kTB - 1) / kTB);
  if (mode == 0)
    k_batched<double, MODE_ANALYSIS><<<grid, 256, 0, ctx->stream>>>(N, P, R, C, M, in, out, ctx->d_rad,
                                                                     scale_by_radius, nullptr, 0);
  else
    k_batched<double, MODE_SYNTH><<<grid, 256, 0, ctx->stream>>>(N, P, R, C, M, in, out, ctx->d_rad,
                                                                  scale_by_radius, sig, half);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_analysis(sps_ctx* ctx, const double* sig, bool fp32) {
  SpsPhase timer(ctx, SPS_PH_SELF);
  const int N = ctx->N, P = ctx->T.P, NR = ctx->T.NR;
  dim3 grid((N + kTB - 1) / kTB, (NR + kTB - 1) / kTB);
#if SPS_SHT_TC
  if (fp32) return sps_launch_sht_tc(ctx, ctx->tcA, 0, sig, ctx->d_coef, 0, nullptr, 0);
#endif
  if (fp32)
    k_batched<float, MODE_ANALYSIS><<<grid, 256, 0, ctx->stream>>>(N, P, NR, 3 * P, ctx->d_anal32, sig,
                                                                    ctx->d_coef, nullptr, 0, nullptr, 0);
  else
    k_batched<double, MODE_ANALYSIS><<<grid, 256, 0, ctx->stream>>>(N, P, NR, 3 * P, ctx->d_anal, sig,
                                                                     ctx->d_coef, nullptr, 0, nullptr, 0);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_self(sps_ctx* ctx, int op, const double* sig, double* out, bool fp32) {
  SpsPhase timer(ctx, SPS_PH_SELF);
  const int N = ctx->N, P = ctx->T.P, NR = ctx->T.NR;
  const bool S = (op == SPS_OP_S);
  dim3 grid((N + kTB - 1) / kTB, (3 * P + kTB - 1) / kTB);
  const int half = (op == SPS_OP_A) ? 1 : 0;
#if SPS_SHT_TC
  if (fp32) return sps_launch_sht_tc(ctx, S ? ctx->tcS : ctx->tcK, 1, ctx->d_coef, out, S ? 1 : 0, sig, half);
#endif
  if (fp32)
    k_batched<float, MODE_SYNTH><<<grid, 256, 0, ctx->stream>>>(
        N, P, 3 * P, NR, S ? ctx->d_synthS32 : ctx->d_synthK32, ctx->d_coef, out, ctx->d_rad, S ? 1 : 0,
        sig, half);
  else
    k_batched<double, MODE_SYNTH><<<grid, 256, 0, ctx->stream>>>(
        N, P, 3 * P, NR, S ? ctx->d_synthS : ctx->d_synthK, ctx->d_coef, out, ctx->d_rad, S ? 1 : 0,
        sig, half);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_near(sps_ctx* ctx, int op, double* out, bool fp32) {
  if (ctx->n_near == 0) return SPS_OK;
  const int N = ctx->N, NR = ctx->T.NR, NC = ctx->T.NC, L = ctx->T.L, E = ctx->T.E;
  const int p = ctx->T.p;
  const bool S = (op == SPS_OP_S);
  {
    SpsPhase timer(ctx, SPS_PH_SELF);
    // field coefficients of every source sphere: fcoef_s = FM coef_s (sparse)
    const sps_ctx::Sparse& fm = S ? ctx->fmS : ctx->fmK;
    SPS_TRY(sps_launch_sparse_rows(ctx, fm, N, ctx->d_coef, NR, ctx->d_fcoef, fm.rows, 0,
                                   fp32 ? ctx->d_fcoef32 : nullptr,
                                   (fp32 && SPS_CLOSE_DW) ? ctx->d_fcoefdw : nullptr));
    (void)NC;
    (void)L;
    (void)E;
    (void)p;
  }
  SpsPhase timer(ctx, S ? SPS_PH_NEAR_S : SPS_PH_NEAR_K);
  // mixed path: FP32 for near entries farther than kCloseRadius source radii,
  // FP64 for the close ones (where the expansion's terms do not decay)
  if (S) {
    if (!fp32) return launch_near_eval<sps::kFieldsS, double>(ctx, 0.0, out);
    if (SPS_NEAR_SRC && SPS_CLOSE_DW) return launch_near_src<sps::kFieldsS>(ctx, out);
    SPS_TRY(launch_near_eval32<sps::kFieldsS>(ctx, out));
    return launch_near_close<sps::kFieldsS>(ctx, out);
  }
  if (!fp32) return launch_near_eval<sps::kFieldsK, double>(ctx, 0.0, out);
  if (SPS_NEAR_SRC && SPS_CLOSE_DW) return launch_near_src<sps::kFieldsK>(ctx, out);
  SPS_TRY(launch_near_eval32<sps::kFieldsK>(ctx, out));
  return launch_near_close<sps::kFieldsK>(ctx, out);
}

#ifndef SPS_MIXED_VSH
#define SPS_MIXED_VSH 1
#endif
#ifndef SPS_MIXED_NEAR
#define SPS_MIXED_NEAR 1
#endif
int sps_layer(sps_ctx* ctx, int op, const double* sig, double* out, bool fp32) {
  ctx->layer_applies += 1;
  // oriented grids: the VSH transforms see each density in its sphere's frame
  // (components Q_i^T sigma), and the self field is rotated back (Q_i u)
  const bool rot = sps_rot(ctx) != nullptr;
  const double* sl = sig;
  if (rot) {
    SPS_TRY(sps_grow(ctx, &ctx->d_sigloc, ctx->cap_sigloc, 3 * (size_t)ctx->NP));
    SPS_TRY(sps_launch_rotate(ctx, sig, ctx->d_sigloc, true));
    sl = ctx->d_sigloc;
  }
  SPS_TRY(sps_launch_analysis(ctx, sl, fp32 && SPS_MIXED_VSH));
  SPS_TRY(sps_launch_self(ctx, op, sl, out, fp32 && SPS_MIXED_VSH));
  if (rot) SPS_TRY(sps_launch_rotate(ctx, out, out, false));
  const int kop = (op == SPS_OP_S) ? SPS_OP_S : SPS_OP_K;
  SPS_TRY(sps_launch_near(ctx, kop, out, fp32 && SPS_MIXED_NEAR));
  SPS_TRY(sps_launch_far(ctx, kop, sig, out, fp32));
  if (op == SPS_OP_A) {
    SPS_TRY(sps_launch_moments(ctx, sig, ctx->d_mom));
    SPS_TRY(sps_launch_add_L(ctx, ctx->d_mom, out));
  }
  return SPS_OK;
}
