// Gradient of a velocity loss with respect to the sphere centres c (radii,
// near lists and quadrature held fixed).  With sigma = rho + zeta, ubar and
// lambda from the adjoint solve (sps_adjoint.cu):
//   dL/dc = ubar . (dS/dc) sigma - lambda . (dK/dc) sigma,
// because the self parts, L, rho and the averages depend only on positions
// relative to each sphere's own centre.  Only cross-sphere terms remain:
//
// Far pairs (target node t on sphere T, source node s on sphere Q):
//   S: f = w_s ubar_t . G(r) sigma_s,        r = x_t - x_s
//   K: f = w_s lambda_t . T(r) : sigma_s n_t
//   dL/dc_T += df/dr (S) or -= (K); dL/dc_Q gets the opposite.  The source-side
//   sums are evaluated as a second target-major pass with the roles of the two
//   vectors swapped (G is even, T is odd, so grad f is odd / even in r):
//   pass A: a = target adjoint, b = w sigma at the source;
//   pass B: a = w sigma at the target, b = adjoint at the source (K: with the
//   source's normal).  dL/dc_Z = sum over nodes of Z of (A_S + B_S - A_K + B_K).
//
// Near pairs (T, Q): the adjoint is contracted with the field first,
//   s(x) = sum_f mu_f(x) F_f(x),  mu_f = C_f . ybar  (as in the reverse evaluation),
// and differentiated with respect to the target position: the fields F_f are
// sums of irregular solid harmonics, whose derivatives shift (n, m) by one
// degree (d_z H_n^m = H_{n+1}^m, (d_x +- i d_y) H_n^m = +-H_{n+1}^{m+-1}),
// plus the explicit dependence of the combination C_f on x.  The per-pair
// sums G_TQ (over the nodes of T) enter T with + and Q with -.
#include <cmath>

#include "sps_internal.cuh"

namespace {

constexpr int kT64 = 128;

// ---------------------------------------------------------------------------
// far pair gradients (FP64)
// ---------------------------------------------------------------------------
// OP S: grad_r [a . G(r) b];  OP K: grad_r [-3/(4 pi) (a.r)(b.r)(c.r)/|r|^5].
// WT: a is multiplied by the target weight; WS: b by the source weight;
// NS: for K, c is the source normal (else the target normal).
template <int OP, bool WT, bool WS, bool NS>
__global__ void __launch_bounds__(kT64) k_far64_grad(int N, int P, const double* __restrict__ X,
                                                     const double* __restrict__ Nr,
                                                     const double* __restrict__ W,
                                                     const double* __restrict__ av,
                                                     const double* __restrict__ bv,
                                                     const int* __restrict__ near_ptr,
                                                     const int* __restrict__ near_idx, double sign,
                                                     double* __restrict__ out) {
  __shared__ double sx[kT64], sy[kT64], sz[kT64], bx[kT64], by[kT64], bz[kT64];
  __shared__ double cx[kT64], cy[kT64], cz[kT64];
  __shared__ int ss[kT64];
  const long long NP = (long long)N * P;
  const long long t = (long long)blockIdx.x * kT64 + threadIdx.x;
  const bool valid = t < NP;
  const long long tt = valid ? t : 0;
  const double tx = X[tt], ty = X[NP + tt], tz = X[2 * NP + tt];
  const double wt = WT ? W[tt] : 1.0;
  const double ax = wt * av[tt], ay = wt * av[NP + tt], az = wt * av[2 * NP + tt];
  double ncx = 0, ncy = 0, ncz = 0;
  if (OP == SPS_OP_K && !NS) {
    ncx = Nr[tt];
    ncy = Nr[NP + tt];
    ncz = Nr[2 * NP + tt];
  }
  const int i = (int)(tt / P);
  int ptr = near_ptr[i];
  const int end = near_ptr[i + 1];
  int cur = -1;
  bool excl = false;
  double gx = 0, gy = 0, gz = 0;
  for (long long t0 = 0; t0 < NP; t0 += kT64) {
    const long long j = t0 + threadIdx.x;
    if (j < NP) {
      const double ws = WS ? W[j] : 1.0;
      sx[threadIdx.x] = X[j];
      sy[threadIdx.x] = X[NP + j];
      sz[threadIdx.x] = X[2 * NP + j];
      bx[threadIdx.x] = ws * bv[j];
      by[threadIdx.x] = ws * bv[NP + j];
      bz[threadIdx.x] = ws * bv[2 * NP + j];
      if (OP == SPS_OP_K && NS) {
        cx[threadIdx.x] = Nr[j];
        cy[threadIdx.x] = Nr[NP + j];
        cz[threadIdx.x] = Nr[2 * NP + j];
      }
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
      const double inv = rsqrt(r2), i2 = inv * inv, i3 = i2 * inv;
      const double ar = ax * rx + ay * ry + az * rz;
      const double br = bx[k] * rx + by[k] * ry + bz[k] * rz;
      if (OP == SPS_OP_S) {
        const double ab = ax * bx[k] + ay * by[k] + az * bz[k];
        const double q = -3.0 * ar * br * i2;
        gx += i3 * (-ab * rx + br * ax + ar * bx[k] + q * rx);
        gy += i3 * (-ab * ry + br * ay + ar * by[k] + q * ry);
        gz += i3 * (-ab * rz + br * az + ar * bz[k] + q * rz);
      } else {
        const double nx = NS ? cx[k] : ncx, ny = NS ? cy[k] : ncy, nz = NS ? cz[k] : ncz;
        const double cr = nx * rx + ny * ry + nz * rz;
        const double i5 = i3 * i2;
        const double q = -5.0 * ar * br * cr * i2;
        gx += i5 * (br * cr * ax + ar * cr * bx[k] + ar * br * nx + q * rx);
        gy += i5 * (br * cr * ay + ar * cr * by[k] + ar * br * ny + q * ry);
        gz += i5 * (br * cr * az + ar * cr * bz[k] + ar * br * nz + q * rz);
      }
    }
    __syncthreads();
  }
  if (valid) {
    const double s = sign * ((OP == SPS_OP_S) ? 1.0 / (8.0 * SPS_PI) : -3.0 / (4.0 * SPS_PI));
    out[t] += s * gx;
    out[NP + t] += s * gy;
    out[2 * NP + t] += s * gz;
  }
}

// per-sphere sums of a 3-plane node field, added into dx (N x 3)
__global__ void k_sphere_sum3(int N, int P, const double* __restrict__ f, double* __restrict__ dx) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  const long long NP = (long long)N * P;
  double m0 = 0, m1 = 0, m2 = 0;
  for (int k = lane; k < P; k += 32) {
    const long long g = (long long)warp * P + k;
    m0 += f[g];
    m1 += f[NP + g];
    m2 += f[2 * NP + g];
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 += __shfl_xor_sync(0xffffffffu, m0, o);
    m1 += __shfl_xor_sync(0xffffffffu, m1, o);
    m2 += __shfl_xor_sync(0xffffffffu, m2, o);
  }
  if (lane == 0) {
    dx[3 * warp] += m0;
    dx[3 * warp + 1] += m1;
    dx[3 * warp + 2] += m2;
  }
}

// ---------------------------------------------------------------------------
// near pair gradients (FP64)
// ---------------------------------------------------------------------------
// signed-m coefficient c_{n,m} of a folded array (m >= 0 entries hold eps_m c)
__device__ __forceinline__ double2 cget(const double* __restrict__ cc, int L, int n, int m) {
  if (n < 0 || n > L || m > n || -m > n) return make_double2(0.0, 0.0);
  const int mm = m < 0 ? -m : m;
  const int e = mm * (L + 1) - mm * (mm - 1) / 2 + (n - mm);
  const double ie = (mm == 0) ? 1.0 : 0.5;
  double re = cc[2 * e] * ie, im = cc[2 * e + 1] * ie;
  if (m < 0) {
    const double sg = (mm & 1) ? -1.0 : 1.0;
    re *= sg;
    im *= -sg;
  }
  return make_double2(re, im);
}

template <int F>
__device__ __forceinline__ void mu_of(double x, double y, double z, double vx, double vy, double vz, double bx,
                                      double by, double bz, double aj, double* lam) {
  const double r2 = x * x + y * y + z * z;
  for (int f = 0; f < F; ++f) lam[f] = 0.0;
  if (F == sps::kFieldsK) {
    auto bil = [](double* o, double px, double py, double pz, double qx, double qy, double qz, double s) {
      o[0] += s * px * qx;
      o[1] += s * (px * qy + py * qx);
      o[2] += s * (px * qz + pz * qx);
      o[3] += s * py * qy;
      o[4] += s * (py * qz + pz * qy);
      o[5] += s * pz * qz;
    };
    bil(lam + 0, bx, by, bz, vx, vy, vz, 2.0);
    const double cx = by * z - bz * y, cy = bz * x - bx * z, cz = bx * y - by * x;
    bil(lam + 6, cx, cy, cz, vx, vy, vz, 1.0);
    const double wx = vy * z - vz * y, wy = vz * x - vx * z, wz = vx * y - vy * x;
    bil(lam + 6, bx, by, bz, wx, wy, wz, 1.0);
    const double xv = x * vx + y * vy + z * vz, bxd = bx * x + by * y + bz * z;
    lam[12] = 2.0 * (xv * bx + bxd * vx);
    lam[13] = 2.0 * (xv * by + bxd * vy);
    lam[14] = 2.0 * (xv * bz + bxd * vz);
    bil(lam + 15, bx, by, bz, vx, vy, vz, 2.0 * r2);
    lam[21] = bxd * vx + xv * bx;
    lam[22] = bxd * vy + xv * by;
    lam[23] = bxd * vz + xv * bz;
    lam[24] = bx * vx + by * vy + bz * vz;
  } else {
    lam[0] = aj * bx;
    lam[1] = aj * by;
    lam[2] = aj * bz;
    lam[3] = aj * (by * z - bz * y);
    lam[4] = aj * (bz * x - bx * z);
    lam[5] = aj * (bx * y - by * x);
    lam[6] = aj * r2 * bx;
    lam[7] = aj * r2 * by;
    lam[8] = aj * r2 * bz;
    lam[9] = aj * (bx * x + by * y + bz * z);
  }
}

constexpr int kMaxE = (sps::kMaxP + 3) * (sps::kMaxP + 4) / 2;

// One block per target sphere T, one thread per node; per near source Q the
// block writes G_TQ = sum over T's nodes of d/dx [ybar . out_Q(x)] into Gp.
template <int F>
__global__ void k_near_grad(int N, int P, int L, int E, const double* __restrict__ pos,
                            const double* __restrict__ rad, const double* __restrict__ X,
                            const double* __restrict__ Nr, const int* __restrict__ near_ptr,
                            const int* __restrict__ near_idx, const double* __restrict__ fcoef,
                            const double* __restrict__ ybar, double* __restrict__ Gp) {
  extern __shared__ __align__(16) double sgc[];
  double* red = sgc + (size_t)E * F * 2;   // blockDim x 3
  const int T = blockIdx.x;
  const long long NP = (long long)N * P;
  const int k = threadIdx.x;
  const bool valid = k < P;
  const long long g = (long long)T * P + (valid ? k : 0);
  const double gx = X[g], gy = X[NP + g], gz = X[2 * NP + g];
  const double vx = Nr[g], vy = Nr[NP + g], vz = Nr[2 * NP + g];
  const double bx = valid ? ybar[g] : 0.0, by = valid ? ybar[NP + g] : 0.0, bz = valid ? ybar[2 * NP + g] : 0.0;
  double cc[2 * kMaxE];   // mu-combined folded coefficients, entries n <= L
  for (int q = near_ptr[T]; q < near_ptr[T + 1]; ++q) {
    const int Q = near_idx[q];
    __syncthreads();
    const double* src = fcoef + (long long)Q * E * F * 2;
    for (int e = threadIdx.x; e < E * F * 2; e += blockDim.x) sgc[e] = src[e];
    __syncthreads();
    const double aj = rad[Q], ia = 1.0 / aj;
    const double x = (gx - pos[3 * Q]) * ia, y = (gy - pos[3 * Q + 1]) * ia, z = (gz - pos[3 * Q + 2]) * ia;
    const double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
    double mu[F];
    mu_of<F>(x, y, z, vx, vy, vz, bx, by, bz, aj, mu);
    // pass 1: field values F_f and combined coefficients cc
    double acc[F];
    for (int f = 0; f < F; ++f) acc[f] = 0.0;
    {
      double dre = 1.0 / sqrt(r2), dim = 0.0;
      int e = 0;
      for (int m = 0; m <= L; ++m) {
        if (m > 0) {
          const double fm = -(2.0 * m - 1.0) * ir2;
          const double re = fm * (x * dre - y * dim), im = fm * (x * dim + y * dre);
          dre = re;
          dim = im;
        }
        double hre = dre, him = dim, pre = 0.0, pim = 0.0;
        for (int n = m; n <= L; ++n, ++e) {
          const double* cf = sgc + e * F * 2;
          double sre = 0.0, sim = 0.0;
#pragma unroll
          for (int f = 0; f < F; ++f) {
            acc[f] = fma(cf[2 * f], hre, fma(-cf[2 * f + 1], him, acc[f]));
            sre = fma(mu[f], cf[2 * f], sre);
            sim = fma(mu[f], cf[2 * f + 1], sim);
          }
          cc[2 * e] = sre;
          cc[2 * e + 1] = sim;
          const double f1 = (2.0 * n + 1.0) * z, f2 = (double)(n * n - m * m);
          const double nre = -(f1 * hre + f2 * pre) * ir2, nim = -(f1 * him + f2 * pim) * ir2;
          pre = hre;
          pim = him;
          hre = nre;
          him = nim;
        }
      }
    }
    // pass 2: gradient of Re sum cc H through the shifted coefficients
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    {
      const int L1 = L + 1;
      double dre = 1.0 / sqrt(r2), dim = 0.0;
      for (int m = 0; m <= L1; ++m) {
        if (m > 0) {
          const double fm = -(2.0 * m - 1.0) * ir2;
          const double re = fm * (x * dre - y * dim), im = fm * (x * dim + y * dre);
          dre = re;
          dim = im;
        }
        double hre = dre, him = dim, pre = 0.0, pim = 0.0;
        const double eps = (m == 0) ? 1.0 : 2.0;
        for (int n = m; n <= L1; ++n) {
          if (n >= 1) {
            const double2 cz = cget(cc, L, n - 1, m);
            const double2 cm = cget(cc, L, n - 1, m - 1), cp = cget(cc, L, n - 1, m + 1);
            // d_z: c(n-1, m); d_x: (c(n-1,m-1) - c(n-1,m+1))/2; d_y: -i (c(n-1,m-1) + c(n-1,m+1))/2
            const double xre = 0.5 * (cm.x - cp.x), xim = 0.5 * (cm.y - cp.y);
            const double yre = 0.5 * (cm.y + cp.y), yim = -0.5 * (cm.x + cp.x);
            d0 += eps * (xre * hre - xim * him);
            d1 += eps * (yre * hre - yim * him);
            d2 += eps * (cz.x * hre - cz.y * him);
          }
          const double f1 = (2.0 * n + 1.0) * z, f2 = (double)(n * n - m * m);
          const double nre = -(f1 * hre + f2 * pre) * ir2, nim = -(f1 * him + f2 * pim) * ir2;
          pre = hre;
          pim = him;
          hre = nre;
          him = nim;
        }
      }
    }
    // explicit dependence of the combination on x (fields held fixed)
    if (F == sps::kFieldsK) {
      const double* HD = acc + 6;
      const double* GL = acc + 12;
      const double* HL = acc + 15;
      const double* GB = acc + 21;
      auto hv = [](const double* H, double a, double b, double c, double& o0, double& o1, double& o2) {
        o0 = H[0] * a + H[1] * b + H[2] * c;
        o1 = H[1] * a + H[3] * b + H[4] * c;
        o2 = H[2] * a + H[4] * b + H[5] * c;
      };
      double hdv0, hdv1, hdv2, hlv0, hlv1, hlv2;
      hv(HD, vx, vy, vz, hdv0, hdv1, hdv2);
      hv(HL, vx, vy, vz, hlv0, hlv1, hlv2);
      const double glv = GL[0] * vx + GL[1] * vy + GL[2] * vz;
      const double gbv = GB[0] * vx + GB[1] * vy + GB[2] * vz;
      const double hdvv[3] = {hdv0, hdv1, hdv2}, hlvv[3] = {hlv0, hlv1, hlv2};
      const double vv[3] = {vx, vy, vz}, xx[3] = {x, y, z}, bb[3] = {bx, by, bz};
      double dd[3];
      for (int kk = 0; kk < 3; ++kk) {
        double ek[3] = {0, 0, 0};
        ek[kk] = 1.0;
        // e_k x (HD v)
        double D0 = ek[1] * hdvv[2] - ek[2] * hdvv[1];
        double D1 = ek[2] * hdvv[0] - ek[0] * hdvv[2];
        double D2 = ek[0] * hdvv[1] - ek[1] * hdvv[0];
        // HD (v x e_k)
        const double wx = vv[1] * ek[2] - vv[2] * ek[1], wy = vv[2] * ek[0] - vv[0] * ek[2],
                     wz = vv[0] * ek[1] - vv[1] * ek[0];
        double o0, o1, o2;
        hv(HD, wx, wy, wz, o0, o1, o2);
        D0 += o0;
        D1 += o1;
        D2 += o2;
        // 2 GL v_k + 2 e_k (GL.v) + 4 x_k HL v + e_k (GB.v) + GB v_k
        D0 += 2 * GL[0] * vv[kk] + 4 * xx[kk] * hlvv[0] + GB[0] * vv[kk];
        D1 += 2 * GL[1] * vv[kk] + 4 * xx[kk] * hlvv[1] + GB[1] * vv[kk];
        D2 += 2 * GL[2] * vv[kk] + 4 * xx[kk] * hlvv[2] + GB[2] * vv[kk];
        const double extra = 2 * glv + gbv;
        if (kk == 0) D0 += extra;
        if (kk == 1) D1 += extra;
        if (kk == 2) D2 += extra;
        dd[kk] = bb[0] * D0 + bb[1] * D1 + bb[2] * D2;
      }
      d0 += dd[0];
      d1 += dd[1];
      d2 += dd[2];
    } else {
      const double* GD = acc + 3;
      const double* GL = acc + 6;
      const double Be = acc[9];
      // d/dx_k of x x GD + r^2 GL + x Be (fields fixed): e_k x GD + 2 x_k GL + e_k Be
      const double xx[3] = {x, y, z};
      for (int kk = 0; kk < 3; ++kk) {
        double ek[3] = {0, 0, 0};
        ek[kk] = 1.0;
        const double D0 = (ek[1] * GD[2] - ek[2] * GD[1]) + 2 * xx[kk] * GL[0] + ek[0] * Be;
        const double D1 = (ek[2] * GD[0] - ek[0] * GD[2]) + 2 * xx[kk] * GL[1] + ek[1] * Be;
        const double D2 = (ek[0] * GD[1] - ek[1] * GD[0]) + 2 * xx[kk] * GL[2] + ek[2] * Be;
        const double v = aj * (bx * D0 + by * D1 + bz * D2);
        if (kk == 0) d0 += v;
        if (kk == 1) d1 += v;
        if (kk == 2) d2 += v;
      }
    }
    // chain rule x~ = (x - c_Q)/a_Q; deterministic block sum (warps, then warp totals)
    double v3[3] = {valid ? d0 * ia : 0.0, valid ? d1 * ia : 0.0, valid ? d2 * ia : 0.0};
    for (int c = 0; c < 3; ++c)
      for (int o = 16; o > 0; o >>= 1) v3[c] += __shfl_xor_sync(0xffffffffu, v3[c], o);
    if ((threadIdx.x & 31) == 0)
      for (int c = 0; c < 3; ++c) red[3 * (threadIdx.x >> 5) + c] = v3[c];
    __syncthreads();
    if (threadIdx.x == 0) {
      double t3[3] = {0.0, 0.0, 0.0};
      for (int wq = 0; wq < (int)(blockDim.x >> 5); ++wq)
        for (int c = 0; c < 3; ++c) t3[c] += red[3 * wq + c];
      for (int c = 0; c < 3; ++c) Gp[3 * (long long)q + c] = t3[c];
    }
  }
}

// dx_T += sum_{Q in near(T)} (GS_TQ - GK_TQ) - (GS_QT - GK_QT)
__global__ void k_near_grad_combine(int N, const int* __restrict__ near_ptr, const int* __restrict__ near_idx,
                                    const double* __restrict__ GS, const double* __restrict__ GK,
                                    double* __restrict__ dx) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= N) return;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int q = near_ptr[T]; q < near_ptr[T + 1]; ++q) {
    const int Q = near_idx[q];
    // index of T in Q's (sorted) list
    int lo = near_ptr[Q], hi = near_ptr[Q + 1] - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (near_idx[mid] < T) lo = mid + 1;
      else hi = mid;
    }
    const int qr = lo;
    a0 += (GS[3 * q] - GK[3 * q]) - (GS[3 * qr] - GK[3 * qr]);
    a1 += (GS[3 * q + 1] - GK[3 * q + 1]) - (GS[3 * qr + 1] - GK[3 * qr + 1]);
    a2 += (GS[3 * q + 2] - GK[3 * q + 2]) - (GS[3 * qr + 2] - GK[3 * qr + 2]);
  }
  dx[3 * T] += a0;
  dx[3 * T + 1] += a1;
  dx[3 * T + 2] += a2;
}

}  // namespace

int sps_geom_gradient(sps_ctx* ctx, const double* ubar, const double* lam, const double* sig, double* dx) {
  SpsPhase timer(ctx, SPS_PH_KRYLOV);
  const int N = ctx->N, P = ctx->T.P, L = ctx->T.L, E = ctx->T.E, NR = ctx->T.NR;
  const long long NP = ctx->NP;
  if (L + 1 > sps::kMaxP + 3) return sps_fail(ctx, SPS_ERR_INVALID_ARG, "order too large for the gradient");
  double* node = ctx->d_r;   // 3 planes of per-node far gradients
  SPS_CUDA(ctx, cudaMemsetAsync(node, 0, sizeof(double) * 3 * NP, ctx->stream));
  SPS_CUDA(ctx, cudaMemsetAsync(dx, 0, sizeof(double) * 3 * N, ctx->stream));
  const int blocks = (int)((NP + kT64 - 1) / kT64);
  // far S: pass A (a = ubar, b = w sigma), pass B (a = w sigma, b = ubar)
  k_far64_grad<SPS_OP_S, false, true, false><<<blocks, kT64, 0, ctx->stream>>>(
      N, P, ctx->d_X, ctx->d_Nrm, ctx->d_W, ubar, sig, ctx->d_near_ptr, ctx->d_near_idx, 1.0, node);
  SPS_LAUNCHED(ctx);
  k_far64_grad<SPS_OP_S, true, false, false><<<blocks, kT64, 0, ctx->stream>>>(
      N, P, ctx->d_X, ctx->d_Nrm, ctx->d_W, sig, ubar, ctx->d_near_ptr, ctx->d_near_idx, 1.0, node);
  SPS_LAUNCHED(ctx);
  // far K: pass A (a = lambda, c = target normal, b = w sigma) with -, pass B
  // (a = w sigma, b = lambda, c = source normal) with +
  k_far64_grad<SPS_OP_K, false, true, false><<<blocks, kT64, 0, ctx->stream>>>(
      N, P, ctx->d_X, ctx->d_Nrm, ctx->d_W, lam, sig, ctx->d_near_ptr, ctx->d_near_idx, -1.0, node);
  SPS_LAUNCHED(ctx);
  k_far64_grad<SPS_OP_K, true, false, true><<<blocks, kT64, 0, ctx->stream>>>(
      N, P, ctx->d_X, ctx->d_Nrm, ctx->d_W, sig, lam, ctx->d_near_ptr, ctx->d_near_idx, 1.0, node);
  SPS_LAUNCHED(ctx);
  k_sphere_sum3<<<(N * 32 + 127) / 128, 128, 0, ctx->stream>>>(N, P, node, dx);
  SPS_LAUNCHED(ctx);
  if (ctx->n_near > 0) {
    // field coefficients of sigma (both field sets), then per-pair gradients
    double *GS = nullptr, *GK = nullptr;
    SPS_CUDA(ctx, cudaMalloc(&GS, sizeof(double) * 3 * (size_t)ctx->n_near));
    SPS_CUDA(ctx, cudaMalloc(&GK, sizeof(double) * 3 * (size_t)ctx->n_near));
    SPS_TRY(sps_launch_analysis(ctx, sig, false));
    const int threads = ((P + 31) / 32) * 32;
    for (int pass = 0; pass < 2; ++pass) {
      const bool S = (pass == 0);
      const sps_ctx::Sparse& fm = S ? ctx->fmS : ctx->fmK;
      SPS_TRY(sps_launch_sparse_rows(ctx, fm, N, ctx->d_coef, NR, ctx->d_fcoef, fm.rows, 0));
      const int F = S ? sps::kFieldsS : sps::kFieldsK;
      const size_t sm = sizeof(double) * ((size_t)E * F * 2 + (size_t)threads * 3);
      if (S) {
        if (sm > 48 * 1024)
          SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_grad<sps::kFieldsS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm));
        k_near_grad<sps::kFieldsS><<<N, threads, sm, ctx->stream>>>(N, P, L, E, ctx->d_pos, ctx->d_rad, ctx->d_X,
                                                                    ctx->d_Nrm, ctx->d_near_ptr, ctx->d_near_idx,
                                                                    ctx->d_fcoef, ubar, GS);
      } else {
        if (sm > 48 * 1024)
          SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_grad<sps::kFieldsK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm));
        k_near_grad<sps::kFieldsK><<<N, threads, sm, ctx->stream>>>(N, P, L, E, ctx->d_pos, ctx->d_rad, ctx->d_X,
                                                                    ctx->d_Nrm, ctx->d_near_ptr, ctx->d_near_idx,
                                                                    ctx->d_fcoef, lam, GK);
      }
      SPS_LAUNCHED(ctx);
    }
    k_near_grad_combine<<<(N + 127) / 128, 128, 0, ctx->stream>>>(N, ctx->d_near_ptr, ctx->d_near_idx, GS, GK, dx);
    SPS_LAUNCHED(ctx);
    SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(GS);
    cudaFree(GK);
  }
  return SPS_OK;
}
