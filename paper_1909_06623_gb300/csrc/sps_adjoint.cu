// Adjoint of the mobility solve: gradients of a velocity loss with respect to
// the applied forces/torques (and, in sps_adjoint_geom.cu, the sphere centres).
//
// The paper has no adjoint; this is the transpose of the discrete forward map
// of Sec. 4.1 (the same quadrature, VSH maps and near lists), so the gradient
// is exact for the discretised problem.  With sigma = rho + zeta,
//   U = E u,  u = S sigma,  zeta = A^{-1} b,  b = -(I/2 + K) rho,  rho = R F,
// and ubar = E^T dL/dU:
//   sbar = S^T ubar,  lambda = A^{-T} sbar (adjoint GMRES),
//   rhobar = sbar - (I/2 + K)^T lambda,  dL/dF = R^T rhobar.
// Transposes of the parts of a layer operator:
//   far S:  (S^T v)_t = w_t sum_s G(x_t - x_s) v_s          (weights at the target)
//   far K:  (K^T v)_t = +3/(4 pi) w_t sum_s r (r.v_s)(r.n_s)/|r|^5, r = x_t - x_s
//           (a double-layer-type sum: T is odd, the normal is the source's)
//   self:   Analysis^T Synthesis^T (host-transposed matrices)
//   near:   Analysis^T FM^T Eval^T, where Eval^T reduces, per source sphere,
//           the target adjoints times the conjugate solid harmonics into field
//           coefficient adjoints (k_near_reverse)
//   L^T:    unweighted moments, weights applied to the broadcast
//   E^T, R^T: the same moment / broadcast kernels with weights swapped.
#include <cmath>
#include <cstring>
#include <vector>

#include "sps_internal.cuh"

namespace {

constexpr int kT64 = 128;

// ---------------------------------------------------------------------------
// far field, transposed (FP64)
// ---------------------------------------------------------------------------
template <int OP>
__global__ void __launch_bounds__(kT64) k_far64_T(int N, int P, const double* __restrict__ X,
                                                  const double* __restrict__ Nr,
                                                  const double* __restrict__ W,
                                                  const double* __restrict__ v,
                                                  const int* __restrict__ near_ptr,
                                                  const int* __restrict__ near_idx,
                                                  double* __restrict__ out) {
  __shared__ double sx[kT64], sy[kT64], sz[kT64], fx[kT64], fy[kT64], fz[kT64];
  __shared__ double nx[kT64], ny[kT64], nz[kT64];
  __shared__ int ss[kT64];
  const long long NP = (long long)N * P;
  const long long t = (long long)blockIdx.x * kT64 + threadIdx.x;
  const bool valid = t < NP;
  const long long tt = valid ? t : 0;
  const double tx = X[tt], ty = X[NP + tt], tz = X[2 * NP + tt];
  const int i = (int)(tt / P);
  int ptr = near_ptr[i];
  const int end = near_ptr[i + 1];
  int cur = -1;
  bool excl = false;
  double ax = 0, ay = 0, az = 0;
  for (long long t0 = 0; t0 < NP; t0 += kT64) {
    const long long j = t0 + threadIdx.x;
    if (j < NP) {
      sx[threadIdx.x] = X[j];
      sy[threadIdx.x] = X[NP + j];
      sz[threadIdx.x] = X[2 * NP + j];
      fx[threadIdx.x] = v[j];
      fy[threadIdx.x] = v[NP + j];
      fz[threadIdx.x] = v[2 * NP + j];
      if (OP == SPS_OP_K) {
        nx[threadIdx.x] = Nr[j];
        ny[threadIdx.x] = Nr[NP + j];
        nz[threadIdx.x] = Nr[2 * NP + j];
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
      const double inv = rsqrt(r2);
      const double rv = rx * fx[k] + ry * fy[k] + rz * fz[k];
      if (OP == SPS_OP_S) {
        const double c = rv * inv * inv * inv;
        ax += fx[k] * inv + c * rx;
        ay += fy[k] * inv + c * ry;
        az += fz[k] * inv + c * rz;
      } else {
        const double rn = rx * nx[k] + ry * ny[k] + rz * nz[k];
        const double i2 = inv * inv;
        const double c = rv * rn * i2 * i2 * inv;
        ax += c * rx;
        ay += c * ry;
        az += c * rz;
      }
    }
    __syncthreads();
  }
  if (valid) {
    const double s = ((OP == SPS_OP_S) ? 1.0 / (8.0 * SPS_PI) : 3.0 / (4.0 * SPS_PI)) * W[t];
    out[t] += s * ax;
    out[NP + t] += s * ay;
    out[2 * NP + t] += s * az;
  }
}

// ---------------------------------------------------------------------------
// near field, reverse evaluation: field-coefficient adjoints of each source
// sphere j from the output adjoints ybar at the nodes of its near partners.
// Forward: F_f(t) = Re sum_e c_f[e] H_e(x_t); out(t) = sum_f C_f(t) F_f(t).
// Reverse: lambda_f(t) = C_f(t) . ybar(t);  cbar_f[e] += lambda_f(t) (Re H_e, -Im H_e).
// ---------------------------------------------------------------------------
constexpr int kRevThreads = 128;
constexpr int kRevChunk = 32;

__device__ __forceinline__ void bil(double* o, double px, double py, double pz, double qx, double qy,
                                    double qz, double s) {
  // d/dH (p^T H q) for symmetric H stored [xx, xy, xz, yy, yz, zz], times s
  o[0] += s * px * qx;
  o[1] += s * (px * qy + py * qx);
  o[2] += s * (px * qz + pz * qx);
  o[3] += s * py * qy;
  o[4] += s * (py * qz + pz * qy);
  o[5] += s * pz * qz;
}

template <int F>
__global__ void __launch_bounds__(kRevThreads) k_near_reverse(
    int N, int P, int L, int E, const double* __restrict__ pos, const double* __restrict__ rad,
    const double* __restrict__ X, const double* __restrict__ Nr, const int* __restrict__ near_ptr,
    const int* __restrict__ near_idx, const double* __restrict__ ybar, double* __restrict__ ebar) {
  extern __shared__ __align__(16) double srev[];
  double* sH = srev;                                   // kRevChunk x E x 2
  double* sLam = sH + (size_t)kRevChunk * E * 2;       // kRevChunk x F
  double* sAcc = sLam + (size_t)kRevChunk * F;         // E x F x 2
  const int j = blockIdx.x;
  const long long NP = (long long)N * P;
  const int EF = E * F;
  for (int q = threadIdx.x; q < 2 * EF; q += blockDim.x) sAcc[q] = 0.0;
  const double aj = rad[j], ia = 1.0 / aj;
  for (int pi = near_ptr[j]; pi < near_ptr[j + 1]; ++pi) {
    const int i = near_idx[pi];   // near is symmetric: i has j among its near sources
    for (int t0 = 0; t0 < P; t0 += kRevChunk) {
      __syncthreads();
      if (threadIdx.x < kRevChunk) {
        const int tl = threadIdx.x;
        double* H = sH + (size_t)tl * E * 2;
        double* lam = sLam + (size_t)tl * F;
        for (int f = 0; f < F; ++f) lam[f] = 0.0;
        if (t0 + tl < P) {
          const long long g = (long long)i * P + t0 + tl;
          const double x = (X[g] - pos[3 * j]) * ia, y = (X[NP + g] - pos[3 * j + 1]) * ia,
                       z = (X[2 * NP + g] - pos[3 * j + 2]) * ia;
          const double bx = ybar[g], by = ybar[NP + g], bz = ybar[2 * NP + g];
          const double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
          if (F == sps::kFieldsK) {
            const double vx = Nr[g], vy = Nr[NP + g], vz = Nr[2 * NP + g];
            // ordering of the 25 fields: HA(6) HD(6) GL(3) HL(6) GB(3) Q(1)
            bil(lam + 0, bx, by, bz, vx, vy, vz, 2.0);
            const double cx = by * z - bz * y, cy = bz * x - bx * z, cz = bx * y - by * x;  // ybar x x
            bil(lam + 6, cx, cy, cz, vx, vy, vz, 1.0);
            const double wx = vy * z - vz * y, wy = vz * x - vx * z, wz = vx * y - vy * x;  // v x x
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
            // ordering of the 10 fields: GA(3) GD(3) GL(3) Be(1); output scaled by a_j
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
              H[2 * e] = hre;
              H[2 * e + 1] = him;
              const double f1 = (2.0 * n + 1.0) * z, f2 = (double)(n * n - m * m);
              const double nre = -(f1 * hre + f2 * pre) * ir2, nim = -(f1 * him + f2 * pim) * ir2;
              pre = hre;
              pim = him;
              hre = nre;
              him = nim;
            }
          }
        } else {
          for (int e = 0; e < 2 * E; ++e) H[e] = 0.0;
        }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < EF; q += blockDim.x) {
        const int e = q / F, f = q - e * F;
        double re = sAcc[2 * q], im = sAcc[2 * q + 1];
        for (int t = 0; t < kRevChunk; ++t) {
          const double l = sLam[t * F + f];
          re = fma(l, sH[((size_t)t * E + e) * 2], re);
          im = fma(-l, sH[((size_t)t * E + e) * 2 + 1], im);
        }
        sAcc[2 * q] = re;
        sAcc[2 * q + 1] = im;
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * EF; q += blockDim.x) ebar[(long long)j * 2 * EF + q] = sAcc[q];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int far_T(sps_ctx* ctx, int op, const double* v, double* out) {
  SpsPhase timer(ctx, op == SPS_OP_S ? SPS_PH_FAR_S : SPS_PH_FAR_K);
  const long long NP = ctx->NP;
  const int blocks = (int)((NP + kT64 - 1) / kT64);
  if (op == SPS_OP_S)
    k_far64_T<SPS_OP_S><<<blocks, kT64, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_X, ctx->d_Nrm, ctx->d_W,
                                                          v, ctx->d_near_ptr, ctx->d_near_idx, out);
  else
    k_far64_T<SPS_OP_K><<<blocks, kT64, 0, ctx->stream>>>(ctx->N, ctx->T.P, ctx->d_X, ctx->d_Nrm, ctx->d_W,
                                                          v, ctx->d_near_ptr, ctx->d_near_idx, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

template <int F>
static int near_reverse(sps_ctx* ctx, const double* ybar) {
  SpsPhase timer(ctx, F == sps::kFieldsK ? SPS_PH_NEAR_K : SPS_PH_NEAR_S);
  const int E = ctx->T.E;
  const size_t sm = sizeof(double) * ((size_t)kRevChunk * E * 2 + (size_t)kRevChunk * F + (size_t)E * F * 2);
  if (sm > 48 * 1024)
    SPS_CUDA(ctx, cudaFuncSetAttribute(k_near_reverse<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_near_reverse<F><<<ctx->N, kRevThreads, sm, ctx->stream>>>(ctx->N, ctx->T.P, ctx->T.L, E, ctx->d_pos, ctx->d_rad,
                                                             ctx->d_X, ctx->d_Nrm, ctx->d_near_ptr,
                                                             ctx->d_near_idx, ybar, ctx->d_ebar);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// out = Op^T v for op S, K or A (= I/2 + K + L), all FP64
int sps_layer_T(sps_ctx* ctx, int op, const double* v, double* out) {
  ctx->layer_applies += 1;
  const int N = ctx->N, NR = ctx->T.NR;
  const bool S = (op == SPS_OP_S);
  // self: coefbar = Synth^T v (times a_s for S)
  SPS_TRY(sps_launch_batched(ctx, 0, S ? ctx->d_synthST : ctx->d_synthKT, NR, 3 * ctx->T.P, v,
                             ctx->d_coefbar, S ? 1 : 0, nullptr, 0));
  // near: coefbar += FM^T Eval^T v
  if (ctx->n_near > 0) {
    if (S) {
      SPS_TRY(near_reverse<sps::kFieldsS>(ctx, v));
      SPS_TRY(sps_launch_sparse_rows(ctx, ctx->fmSt, N, ctx->d_ebar, ctx->fmSt.cols, ctx->d_coefbar, NR, 1));
    } else {
      SPS_TRY(near_reverse<sps::kFieldsK>(ctx, v));
      SPS_TRY(sps_launch_sparse_rows(ctx, ctx->fmKt, N, ctx->d_ebar, ctx->fmKt.cols, ctx->d_coefbar, NR, 1));
    }
  }
  // out = Analysis^T coefbar (+ v/2 for A)
  SPS_TRY(sps_launch_batched(ctx, 1, ctx->d_analT, 3 * ctx->T.P, NR, ctx->d_coefbar, out, 0,
                             op == SPS_OP_A ? v : nullptr, op == SPS_OP_A ? 1 : 0));
  if (ctx->prm.precision == SPS_MIXED)
    SPS_TRY(sps_launch_far_T32(ctx, S ? SPS_OP_S : SPS_OP_K, v, out));
  else
    SPS_TRY(far_T(ctx, S ? SPS_OP_S : SPS_OP_K, v, out));
  if (op == SPS_OP_A) {
    // L^T: unweighted moments, weighted broadcast
    SPS_TRY(sps_launch_moments_w(ctx, v, ctx->d_mom, false));
    SPS_TRY(sps_launch_add_L_w(ctx, ctx->d_mom, out, true));
  }
  return SPS_OK;
}

extern "C" int sps_layer_apply_transpose(sps_ctx* ctx, int op, const double* v, double* out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!ctx->have_geom) return sps_fail(ctx, SPS_ERR_NO_GEOMETRY, "no geometry");
  if (op < SPS_OP_S || op > SPS_OP_A || !v || !out)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "layer_apply_transpose: bad argument");
  if (ctx->rot_n > 0)
    return sps_fail(ctx, SPS_ERR_INVALID_ARG, "layer_apply_transpose: not available with grid orientations");
  SPS_TRY(sps_layer_T(ctx, op, v, out));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}
