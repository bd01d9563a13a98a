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
#include "sps_dw.cuh"
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
// FP32 kernel (mixed precision)
//
// Coordinates: every node is stored as its offset from its own sphere centre
// (FP32), every centre as an FP32 pair hi + lo (hi = fl(c), lo = fl(c - hi)).
// For target t on sphere i and source s on sphere j the pair vector is
//   r = ((hi_i - hi_j) + (lo_i + d_t - lo_j)) - d_s,
// whose rounding error is relative to |r|, not to the absolute coordinates.
// Sources are staged in shared memory a few whole spheres at a time; each
// (target, source sphere) partial sum is formed in FP32 and added into a
// Kahan-compensated running sum unless sphere j is i or a near neighbour of i
// (a select, so the r = 0 self pair never reaches the sum).  Two targets share
// one packed FP32x2 register pair (fma.rn.f32x2 and friends), so one issued
// instruction does the arithmetic of two pair terms.
// Work items (target block, source split) are taken from an atomic counter by
// a persistent grid; each item writes its own partial sums, which a second
// kernel adds in a fixed order: results do not depend on scheduling.
// ---------------------------------------------------------------------------
#ifndef SPS_FAR_NPAIR
#define SPS_FAR_NPAIR 2
#endif
#ifndef SPS_FAR_THREADS
#define SPS_FAR_THREADS 128
#endif
#ifndef SPS_FAR_MINB
#define SPS_FAR_MINB 3
#endif
constexpr int kT32 = SPS_FAR_THREADS;         // threads per block
constexpr int kNPair = SPS_FAR_NPAIR;         // target pairs per thread
#ifndef SPS_FAR_PACKED
#define SPS_FAR_PACKED 2
#endif
// 1: the Kahan running sums (touched once per source sphere) live in shared
// memory instead of registers
// source nodes per unrolled inner-loop iteration
#ifndef SPS_FAR_UNROLL
#define SPS_FAR_UNROLL 4
#endif
constexpr int kUnroll = SPS_FAR_UNROLL;
#ifndef SPS_FAR_KSMEM
#define SPS_FAR_KSMEM 0
#endif
// pairs q < kPacked use packed FP32x2 instructions, the others scalar FP32
// (measured on GB300: all-packed is fastest; the scalar path is kept for
// tuning on other parts).
constexpr int kPacked = SPS_FAR_PACKED;
constexpr int kOpKT = 3;   // transposed traction (double-layer-type sum, source normals)
static_assert(kPacked == kNPair, "the transposed traction uses the packed path only");
constexpr int kTPB32 = kT32 * 2 * kNPair;     // targets per block
constexpr int kChunkNodes = 512;              // staged source nodes (whole spheres)

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Traction kernels take |r|^-5 from the SFU as 2^(-2.5 log2 |r|^2) instead of
// rsqrt and three multiplies: the FMA pipe (the binding unit) then issues 18
// instead of 20 packed operations per pair.  Measured on 1,000 spheres at
// p = 6: 7.25 -> 6.02 ms per traction application, operator error against FP64
// 3.1e-7 (3.0e-7 before); SPS_FAR_EXP2 = 0 restores the rsqrt form.
#ifndef SPS_FAR_EXP2
#define SPS_FAR_EXP2 1
#endif
// SFU base-2 logarithm and power (PTX lg2.approx / ex2.approx)
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int OP>
__global__ void __launch_bounds__(kT32, SPS_FAR_MINB) k_far32(
    int N, int P, int spc, int n_tb, int n_items, int n_splits,
    const float* __restrict__ rel,    // 3 planes NP: node - own centre
    const float* __restrict__ nrm,    // 3 planes NP
    const float* __restrict__ wsig,   // 3 planes NP: w * sigma
    const float* __restrict__ chi,    // N x 3 centre hi
    const float* __restrict__ clo,    // N x 3 centre lo
    const int* __restrict__ near_ptr, const int* __restrict__ near_idx,
    int* __restrict__ work, double* __restrict__ part) {
  extern __shared__ __align__(16) float4 sdyn[];
  const long long NP = (long long)N * P;
  const int cap = spc * P;                     // nodes per staged chunk
  float4* sA = sdyn;                           // (-dx, -dx, -dy, -dy)
  float4* sB = sA + cap;                       // (-dz, -dz, wx, wx)
  float4* sC = sB + cap;                       // (wy, wy, wz, wz)
  // OP_KT (transposed traction): source normals (nx, nx, ny, ny), (nz, nz, -, -)
  float4* sD = sC + cap;
  float4* sE = sD + (OP == kOpKT ? cap : 0);
  float* sh = reinterpret_cast<float*>(sE + (OP == kOpKT ? cap : 0));  // spc x 6: hi, lo
  // per-thread target state kept out of registers: hi, lo + offset (6 per target)
  __shared__ float sEF[6 * 2 * kNPair][kT32];
  __shared__ int sX[3 * 2 * kNPair][kT32];        // sphere, near pointer, near end
#if SPS_FAR_KSMEM
  __shared__ float2 sKS[6 * kNPair][kT32];        // running sums and compensations
#endif
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const int tb = item % n_tb, sp = item / n_tb;
    const int j_begin = (int)((long long)N * sp / n_splits);
    const int j_end = (int)((long long)N * (sp + 1) / n_splits);
    // ---- targets of this thread: lanes (2q, 2q+1) of pair q
    const long long base = (long long)tb * kTPB32 + threadIdx.x;
    float2 nx[kNPair], ny[kNPair], nz[kNPair];
#if !SPS_FAR_KSMEM
    float2 sx[kNPair], sy[kNPair], sz[kNPair], cx[kNPair], cy[kNPair], cz[kNPair];
#endif
#pragma unroll
    for (int q = 0; q < kNPair; ++q) {
      float n[2][3];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int l = 2 * q + h;
        const long long t = base + (long long)l * kT32;
        const long long tt = t < NP ? t : NP - 1;
        const int i = (int)(tt / P);
        for (int c = 0; c < 3; ++c) {
          sEF[6 * l + c][threadIdx.x] = chi[3 * i + c];
          sEF[6 * l + 3 + c][threadIdx.x] = clo[3 * i + c] + rel[c * NP + tt];
          n[h][c] = (OP == SPS_OP_K) ? nrm[c * NP + tt] : 0.f;   // target normal (K)
        }
        // first near neighbour not below j_begin
        int a = near_ptr[i];
        const int b = near_ptr[i + 1];
        while (a < b && near_idx[a] < j_begin) ++a;
        sX[3 * l][threadIdx.x] = i;
        sX[3 * l + 1][threadIdx.x] = a;
        sX[3 * l + 2][threadIdx.x] = b;
      }
      nx[q] = make_float2(n[0][0], n[1][0]);
      ny[q] = make_float2(n[0][1], n[1][1]);
      nz[q] = make_float2(n[0][2], n[1][2]);
#if SPS_FAR_KSMEM
      for (int c = 0; c < 6; ++c) sKS[6 * q + c][threadIdx.x] = make_float2(0.f, 0.f);
#else
      sx[q] = sy[q] = sz[q] = cx[q] = cy[q] = cz[q] = make_float2(0.f, 0.f);
#endif
    }
    // ---- source spheres, staged spc at a time
    for (int j0 = j_begin; j0 < j_end; j0 += spc) {
      const int ns = min(spc, j_end - j0);
      const int nn = ns * P;
      const long long g0 = (long long)j0 * P;
      __syncthreads();
      for (int k = threadIdx.x; k < nn; k += kT32) {
        const long long g = g0 + k;
        const float dx = -rel[g], dy = -rel[NP + g], dz = -rel[2 * NP + g];   // negated offsets
        const float wx = wsig[g], wy = wsig[NP + g], wz = wsig[2 * NP + g];
        sA[k] = make_float4(dx, dx, dy, dy);
        sB[k] = make_float4(dz, dz, wx, wx);
        sC[k] = make_float4(wy, wy, wz, wz);
        if (OP == kOpKT) {
          const float mx = nrm[g], my = nrm[NP + g], mz = nrm[2 * NP + g];
          sD[k] = make_float4(mx, mx, my, my);
          sE[k] = make_float4(mz, mz, 0.f, 0.f);
        }
      }
      for (int k = threadIdx.x; k < ns * 6; k += kT32) {
        const int js = k / 6, c = k % 6;
        sh[k] = (c < 3) ? chi[3 * (j0 + js) + c] : clo[3 * (j0 + js) + c - 3];
      }
      __syncthreads();
      for (int js = 0; js < ns; ++js) {
        const int j = j0 + js;
        const float hx = sh[6 * js], hy = sh[6 * js + 1], hz = sh[6 * js + 2];
        const float lx = sh[6 * js + 3], ly = sh[6 * js + 4], lz = sh[6 * js + 5];
        float2 Dx[kNPair], Dy[kNPair], Dz[kNPair], ax[kNPair], ay[kNPair], az[kNPair];
#pragma unroll
        for (int q = 0; q < kNPair; ++q) {
          const int l0 = 12 * q, l1 = 12 * q + 6;
          const float2 Ex = make_float2(sEF[l0][threadIdx.x], sEF[l1][threadIdx.x]);
          const float2 Ey = make_float2(sEF[l0 + 1][threadIdx.x], sEF[l1 + 1][threadIdx.x]);
          const float2 Ez = make_float2(sEF[l0 + 2][threadIdx.x], sEF[l1 + 2][threadIdx.x]);
          const float2 Fx = make_float2(sEF[l0 + 3][threadIdx.x], sEF[l1 + 3][threadIdx.x]);
          const float2 Fy = make_float2(sEF[l0 + 4][threadIdx.x], sEF[l1 + 4][threadIdx.x]);
          const float2 Fz = make_float2(sEF[l0 + 5][threadIdx.x], sEF[l1 + 5][threadIdx.x]);
          Dx[q] = __fadd2_rn(__fadd2_rn(Ex, f2(-hx)), __fadd2_rn(Fx, f2(-lx)));
          Dy[q] = __fadd2_rn(__fadd2_rn(Ey, f2(-hy)), __fadd2_rn(Fy, f2(-ly)));
          Dz[q] = __fadd2_rn(__fadd2_rn(Ez, f2(-hz)), __fadd2_rn(Fz, f2(-lz)));
          ax[q] = ay[q] = az[q] = make_float2(0.f, 0.f);
        }
        const float4* A = sA + js * P;
        const float4* B = sB + js * P;
        const float4* C = sC + js * P;
        const float4* D = sD + js * P;
        const float4* Es = sE + js * P;
        (void)D;
        (void)Es;
#pragma unroll kUnroll
        for (int k = 0; k < P; ++k) {
          const float4 a4 = A[k], b4 = B[k], c4 = C[k];
          const float2 sxx = make_float2(a4.x, a4.y), syy = make_float2(a4.z, a4.w);
          const float2 szz = make_float2(b4.x, b4.y), wxx = make_float2(b4.z, b4.w);
          const float2 wyy = make_float2(c4.x, c4.y), wzz = make_float2(c4.z, c4.w);
#pragma unroll
          for (int q = 0; q < kNPair; ++q) {
            if (q < kPacked) {
              const float2 rx = __fadd2_rn(Dx[q], sxx);
              const float2 ry = __fadd2_rn(Dy[q], syy);
              const float2 rz = __fadd2_rn(Dz[q], szz);
              const float2 r2 = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
              const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
              const float2 rs = __ffma2_rn(rz, wzz, __ffma2_rn(ry, wyy, __fmul2_rn(rx, wxx)));
              const float2 i2 = __fmul2_rn(inv, inv);
              if (OP == SPS_OP_S) {
                const float2 cc = __fmul2_rn(__fmul2_rn(rs, i2), inv);
                ax[q] = __ffma2_rn(wxx, inv, __ffma2_rn(cc, rx, ax[q]));
                ay[q] = __ffma2_rn(wyy, inv, __ffma2_rn(cc, ry, ay[q]));
                az[q] = __ffma2_rn(wzz, inv, __ffma2_rn(cc, rz, az[q]));
              } else {
                float2 rn;
                if (OP == kOpKT) {
                  const float4 d4 = D[k], e4 = Es[k];
                  rn = __ffma2_rn(rz, make_float2(e4.x, e4.y),
                                  __ffma2_rn(ry, make_float2(d4.z, d4.w), __fmul2_rn(rx, make_float2(d4.x, d4.y))));
                } else {
                  rn = __ffma2_rn(rz, nz[q], __ffma2_rn(ry, ny[q], __fmul2_rn(rx, nx[q])));
                }
#if SPS_FAR_EXP2
                // |r|^-5 = 2^(-2.5 log2 |r|^2) on the SFU: one packed multiply on the FMA
                // pipe instead of three
                const float2 lg = make_float2(lg2_approx(r2.x), lg2_approx(r2.y));
                const float2 tt = __fmul2_rn(lg, f2(-2.5f));
                const float2 i5 = make_float2(ex2_approx(tt.x), ex2_approx(tt.y));
#else
                const float2 i5 = __fmul2_rn(__fmul2_rn(i2, i2), inv);
#endif
                const float2 cc = __fmul2_rn(__fmul2_rn(rs, rn), i5);
                ax[q] = __ffma2_rn(cc, rx, ax[q]);
                ay[q] = __ffma2_rn(cc, ry, ay[q]);
                az[q] = __ffma2_rn(cc, rz, az[q]);
              }
            } else {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float dX = h ? Dx[q].y : Dx[q].x, dY = h ? Dy[q].y : Dy[q].x;
                const float dZ = h ? Dz[q].y : Dz[q].x;
                const float rx = dX + sxx.x, ry = dY + syy.x, rz = dZ + szz.x;
                const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                const float inv = rsqrtf(r2);
                const float rs = fmaf(rz, wzz.x, fmaf(ry, wyy.x, rx * wxx.x));
                const float i2 = inv * inv;
                float bx = h ? ax[q].y : ax[q].x, by = h ? ay[q].y : ay[q].x;
                float bz = h ? az[q].y : az[q].x;
                if (OP == SPS_OP_S) {
                  const float cc = rs * i2 * inv;
                  bx = fmaf(wxx.x, inv, fmaf(cc, rx, bx));
                  by = fmaf(wyy.x, inv, fmaf(cc, ry, by));
                  bz = fmaf(wzz.x, inv, fmaf(cc, rz, bz));
                } else {
                  const float vx = h ? nx[q].y : nx[q].x, vy = h ? ny[q].y : ny[q].x;
                  const float vz = h ? nz[q].y : nz[q].x;
                  const float rn = fmaf(rz, vz, fmaf(ry, vy, rx * vx));
                  const float cc = (rs * rn) * (i2 * i2 * inv);
                  bx = fmaf(cc, rx, bx);
                  by = fmaf(cc, ry, by);
                  bz = fmaf(cc, rz, bz);
                }
                if (h) {
                  ax[q].y = bx; ay[q].y = by; az[q].y = bz;
                } else {
                  ax[q].x = bx; ay[q].x = by; az[q].x = bz;
                }
              }
            }
          }
        }
        // fold the sphere's partial sums unless j is excluded for the target
#pragma unroll
        for (int q = 0; q < kNPair; ++q) {
          bool ex[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int l = 2 * q + h;
            int pt = sX[3 * l + 1][threadIdx.x];
            const int pe = sX[3 * l + 2][threadIdx.x];
            while (pt < pe && near_idx[pt] < j) ++pt;
            sX[3 * l + 1][threadIdx.x] = pt;
            ex[h] = (j == sX[3 * l][threadIdx.x]) || (pt < pe && near_idx[pt] == j);
          }
          const float2 zx = make_float2(ex[0] ? 0.f : ax[q].x, ex[1] ? 0.f : ax[q].y);
          const float2 zy = make_float2(ex[0] ? 0.f : ay[q].x, ex[1] ? 0.f : ay[q].y);
          const float2 zz = make_float2(ex[0] ? 0.f : az[q].x, ex[1] ? 0.f : az[q].y);
#if SPS_FAR_KSMEM
          float2 Sx = sKS[6 * q][threadIdx.x], Sy = sKS[6 * q + 1][threadIdx.x], Sz = sKS[6 * q + 2][threadIdx.x];
          float2 Cx = sKS[6 * q + 3][threadIdx.x], Cy = sKS[6 * q + 4][threadIdx.x], Cz = sKS[6 * q + 5][threadIdx.x];
#else
          float2 &Sx = sx[q], &Sy = sy[q], &Sz = sz[q], &Cx = cx[q], &Cy = cy[q], &Cz = cz[q];
#endif
          float2 y, t;
          y = __fadd2_rn(zx, make_float2(-Cx.x, -Cx.y));
          t = __fadd2_rn(Sx, y);
          Cx = __fadd2_rn(__fadd2_rn(t, make_float2(-Sx.x, -Sx.y)), make_float2(-y.x, -y.y));
          Sx = t;
          y = __fadd2_rn(zy, make_float2(-Cy.x, -Cy.y));
          t = __fadd2_rn(Sy, y);
          Cy = __fadd2_rn(__fadd2_rn(t, make_float2(-Sy.x, -Sy.y)), make_float2(-y.x, -y.y));
          Sy = t;
          y = __fadd2_rn(zz, make_float2(-Cz.x, -Cz.y));
          t = __fadd2_rn(Sz, y);
          Cz = __fadd2_rn(__fadd2_rn(t, make_float2(-Sz.x, -Sz.y)), make_float2(-y.x, -y.y));
          Sz = t;
#if SPS_FAR_KSMEM
          sKS[6 * q][threadIdx.x] = Sx;
          sKS[6 * q + 1][threadIdx.x] = Sy;
          sKS[6 * q + 2][threadIdx.x] = Sz;
          sKS[6 * q + 3][threadIdx.x] = Cx;
          sKS[6 * q + 4][threadIdx.x] = Cy;
          sKS[6 * q + 5][threadIdx.x] = Cz;
#endif
        }
      }
    }
    // ---- this item's partial sums
    double* o = part + (long long)sp * 3 * NP;
#pragma unroll
    for (int q = 0; q < kNPair; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long t = base + (long long)(2 * q + h) * kT32;
        if (t < NP) {
#if SPS_FAR_KSMEM
          const float2 Sx = sKS[6 * q][threadIdx.x], Sy = sKS[6 * q + 1][threadIdx.x], Sz = sKS[6 * q + 2][threadIdx.x];
          const float2 Cx = sKS[6 * q + 3][threadIdx.x], Cy = sKS[6 * q + 4][threadIdx.x], Cz = sKS[6 * q + 5][threadIdx.x];
#else
          const float2 Sx = sx[q], Sy = sy[q], Sz = sz[q], Cx = cx[q], Cy = cy[q], Cz = cz[q];
#endif
          const float vx = h ? Sx.y : Sx.x, kx = h ? Cx.y : Cx.x;
          const float vy = h ? Sy.y : Sy.x, ky = h ? Cy.y : Cy.x;
          const float vz = h ? Sz.y : Sz.x, kz = h ? Cz.y : Cz.x;
          o[t] = (double)vx - (double)kx;
          o[NP + t] = (double)vy - (double)ky;
          o[2 * NP + t] = (double)vz - (double)kz;
        }
      }
  }
}

__global__ void k_reduce_parts(long long n3, int splits, const double* __restrict__ part,
                               double scale, const double* __restrict__ Wt, double* __restrict__ out) {
  const long long NP = n3 / 3;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n3;
       g += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += part[k * n3 + g];
    out[g] += scale * (Wt ? Wt[g % NP] : 1.0) * s;
  }
}

// w * sigma in FP32 (3 planes), the source strengths of the far field
__global__ void k_wsig32(long long NP, const double* __restrict__ sig, const double* __restrict__ W,
                         float* __restrict__ out) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < 3 * NP;
       g += (long long)gridDim.x * blockDim.x)
    out[g] = (float)((W ? W[g % NP] : 1.0) * sig[g]);
}

// ---------------------------------------------------------------------------
// Double-float kernel: FP64-accurate far field on the FP32 pipe
//
// The same sums as k_far64 with every pair term in double-float arithmetic
// (sps_dw.cuh: about 2^-46 relative per operation) and FP64 accumulation of
// the per-sphere partial sums, so that the result agrees with the FP64
// kernel to about 1e-13 of its size while the arithmetic runs on the FP32
// pipe, which GB300 executes about 64 times faster than FP64.  It evaluates
// the FP64-class operator applications of the mixed path's iterative
// refinement (residual and final velocity) and of the SPS_FP64_DW path.
//
// For target t on sphere i and source s on sphere j:
//   r = E_ij(t) - l_s,  E_ij(t) = (c_i - c_j) + l_t,  l = node - own centre,
// with E formed in FP64 once per (target, source sphere) and split into a
// double-float, and l_s, w_s sigma_s staged in shared memory as double-floats
// (prepared per application by k_dw_src).  1/|r| comes from the SFU estimate
// and one double-float Newton step.  Partial sums over a source sphere are
// folded into FP64 unless j is i or a near neighbour of i; work items (target
// block, source split) come from an atomic queue and write FP64 partials that
// k_reduce_parts adds in a fixed order.
// ---------------------------------------------------------------------------
using namespace sps_dw;
constexpr int kTdw = 128;          // threads per block, one target each
constexpr int kChunkDw = 512;      // staged source nodes (whole spheres)

// per node: (-l_x, -l_y) hi/lo, (-l_z, (w sigma)_x) hi/lo, (w sigma)_y, _z hi/lo
__global__ void k_dw_src(int N, int P, const double* __restrict__ pos, const double* __restrict__ X,
                         const double* __restrict__ W, const double* __restrict__ sig,
                         float4* __restrict__ A, float4* __restrict__ B, float4* __restrict__ C) {
  const long long NP = (long long)N * P;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NP;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / P);
    const dw lx = dw_of(pos[3 * s] - X[g]), ly = dw_of(pos[3 * s + 1] - X[NP + g]),
             lz = dw_of(pos[3 * s + 2] - X[2 * NP + g]);
    const double w = W[g];
    const dw fx = dw_of(w * sig[g]), fy = dw_of(w * sig[NP + g]), fz = dw_of(w * sig[2 * NP + g]);
    A[g] = make_float4(lx.h, lx.l, ly.h, ly.l);
    B[g] = make_float4(lz.h, lz.l, fx.h, fx.l);
    C[g] = make_float4(fy.h, fy.l, fz.h, fz.l);
  }
}

template <int OP>
__global__ void __launch_bounds__(kTdw) k_far_dw(int N, int P, int spc, int n_tb, int n_items, int n_splits,
                                                 const double* __restrict__ pos, const double* __restrict__ X,
                                                 const double* __restrict__ Nr, const float4* __restrict__ gA,
                                                 const float4* __restrict__ gB, const float4* __restrict__ gC,
                                                 const int* __restrict__ near_ptr,
                                                 const int* __restrict__ near_idx, int* __restrict__ work,
                                                 double* __restrict__ part) {
  extern __shared__ __align__(16) float4 sdw[];
  const long long NP = (long long)N * P;
  const int cap = spc * P;
  float4* sA = sdw;
  float4* sB = sA + cap;
  float4* sC = sB + cap;
  double* sc = reinterpret_cast<double*>(sC + cap);   // spc x 3 centres
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const int tb = item % n_tb, sp = item / n_tb;
    const int j_begin = (int)((long long)N * sp / n_splits);
    const int j_end = (int)((long long)N * (sp + 1) / n_splits);
    const long long t = (long long)tb * kTdw + threadIdx.x;
    const long long tt = t < NP ? t : NP - 1;
    const int i = (int)(tt / P);
    const double cx = pos[3 * i], cy = pos[3 * i + 1], cz = pos[3 * i + 2];
    const double ltx = X[tt] - cx, lty = X[NP + tt] - cy, ltz = X[2 * NP + tt] - cz;
    dw nx(0.f, 0.f), ny(0.f, 0.f), nz(0.f, 0.f);
    if (OP == SPS_OP_K) {
      nx = dw_of(Nr[tt]);
      ny = dw_of(Nr[NP + tt]);
      nz = dw_of(Nr[2 * NP + tt]);
    }
    int pt = near_ptr[i];
    const int pe = near_ptr[i + 1];
    while (pt < pe && near_idx[pt] < j_begin) ++pt;
    double ox = 0.0, oy = 0.0, oz = 0.0;
    for (int j0 = j_begin; j0 < j_end; j0 += spc) {
      const int ns = min(spc, j_end - j0);
      const int nn = ns * P;
      const long long g0 = (long long)j0 * P;
      __syncthreads();
      for (int k = threadIdx.x; k < nn; k += kTdw) {
        sA[k] = gA[g0 + k];
        sB[k] = gB[g0 + k];
        sC[k] = gC[g0 + k];
      }
      for (int k = threadIdx.x; k < 3 * ns; k += kTdw) sc[k] = pos[3 * j0 + k];
      __syncthreads();
      for (int js = 0; js < ns; ++js) {
        const int j = j0 + js;
        while (pt < pe && near_idx[pt] < j) ++pt;
        const bool excl = (j == i) || (pt < pe && near_idx[pt] == j);
        if (excl) continue;          // (the whole sphere's terms are skipped)
        const dw Ex = dw_of((cx - sc[3 * js]) + ltx), Ey = dw_of((cy - sc[3 * js + 1]) + lty),
                 Ez = dw_of((cz - sc[3 * js + 2]) + ltz);
        dw ax(0.f, 0.f), ay(0.f, 0.f), az(0.f, 0.f);
        const float4* A = sA + js * P;
        const float4* B = sB + js * P;
        const float4* C = sC + js * P;
#pragma unroll 2
        for (int k = 0; k < P; ++k) {
          const float4 a4 = A[k], b4 = B[k], c4 = C[k];
          const dw rx = dw_add_u(Ex, dw(a4.x, a4.y));
          const dw ry = dw_add_u(Ey, dw(a4.z, a4.w));
          const dw rz = dw_add_u(Ez, dw(b4.x, b4.y));
          const dw wx(b4.z, b4.w), wy(c4.x, c4.y), wz(c4.z, c4.w);
          const dw r2 = dw_norm(dw_add_u(dw_add_u(dw_sqr_u(rx), dw_sqr_u(ry)), dw_sqr_u(rz)));
          const dw y = dw_rsqrt(r2);
          const dw rs = dw_norm(dw_add_u(dw_add_u(dw_mul_u(rx, wx), dw_mul_u(ry, wy)), dw_mul_u(rz, wz)));
          if (OP == SPS_OP_S) {
            // w G sigma (8 pi) = w sigma / |r| + r (r . w sigma) / |r|^3
            const dw y3 = dw_norm(dw_mul_u(dw_mul_u(y, y), y));
            const dw c = dw_norm(dw_mul_u(rs, y3));
            ax = dw_add_u(ax, dw_add_u(dw_mul_u(wx, y), dw_mul_u(c, rx)));
            ay = dw_add_u(ay, dw_add_u(dw_mul_u(wy, y), dw_mul_u(c, ry)));
            az = dw_add_u(az, dw_add_u(dw_mul_u(wz, y), dw_mul_u(c, rz)));
          } else {
            // w T : sigma n (-4 pi / 3) = r (r . w sigma)(r . n) / |r|^5
            const dw rn = dw_norm(dw_add_u(dw_add_u(dw_mul_u(rx, nx), dw_mul_u(ry, ny)), dw_mul_u(rz, nz)));
            const dw y2 = dw_mul_u(y, y);
            const dw y5 = dw_norm(dw_mul_u(dw_mul_u(y2, y2), y));
            const dw c = dw_norm(dw_mul_u(dw_norm(dw_mul_u(rs, rn)), y5));
            ax = dw_add_u(ax, dw_mul_u(c, rx));
            ay = dw_add_u(ay, dw_mul_u(c, ry));
            az = dw_add_u(az, dw_mul_u(c, rz));
          }
        }
        ox += dw_val(ax);
        oy += dw_val(ay);
        oz += dw_val(az);
      }
    }
    if (t < NP) {
      double* o = part + (long long)sp * 3 * NP;
      o[t] = ox;
      o[NP + t] = oy;
      o[2 * NP + t] = oz;
    }
  }
}

}  // namespace

// double-float far sum (op SPS_OP_S or SPS_OP_K), FP64 result added to out
static int far_dw_run(sps_ctx* ctx, int op, const double* sig, double* out, int phase) {
  const long long NP = ctx->NP;
  const int P = ctx->T.P, N = ctx->N;
  const long long n3 = 3 * NP;
  SPS_TRY(sps_grow(ctx, &ctx->d_dwsrc, ctx->cap_dwsrc, (size_t)3 * NP));
  float4 *A = ctx->d_dwsrc, *B = A + NP, *C = B + NP;
  {
    SpsPhase timer(ctx, SPS_PH_FAR_AUX);
    k_dw_src<<<(int)std::min<long long>((NP + 255) / 256, 4096), 256, 0, ctx->stream>>>(
        N, P, ctx->d_pos, ctx->d_X, ctx->d_W, sig, A, B, C);
    SPS_LAUNCHED(ctx);
  }
  const int spc = std::max(1, kChunkDw / P);
  const size_t smem = (size_t)3 * spc * P * sizeof(float4) + (size_t)spc * 3 * sizeof(double);
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  auto kern = (op == SPS_OP_S) ? k_far_dw<SPS_OP_S> : k_far_dw<SPS_OP_K>;
  if (smem > 48 * 1024)
    SPS_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTdw, smem);
  const int resident = std::max(1, per_sm) * std::max(1, sms);
  const int n_tb = (int)((NP + kTdw - 1) / kTdw);
  int splits = (int)std::min<long long>(std::max(1, (8 * resident + n_tb - 1) / n_tb), (long long)N);
  splits = std::min(splits, 64);
  const int n_items = n_tb * splits;
  const int grid = std::min(n_items, resident);
  SPS_TRY(sps_grow(ctx, &ctx->d_part, ctx->cap_part, (size_t)splits * n3 + 1));
  int* d_work = reinterpret_cast<int*>(ctx->d_part + (size_t)splits * n3);
  SPS_CUDA(ctx, cudaMemsetAsync(d_work, 0, sizeof(int), ctx->stream));
  {
    SpsPhase timer(ctx, phase);
    kern<<<grid, kTdw, smem, ctx->stream>>>(N, P, spc, n_tb, n_items, splits, ctx->d_pos, ctx->d_X, ctx->d_Nrm,
                                            A, B, C, ctx->d_near_ptr, ctx->d_near_idx, d_work, ctx->d_part);
    SPS_LAUNCHED(ctx);
  }
  SpsPhase timer(ctx, SPS_PH_FAR_AUX);
  const double scale = (op == SPS_OP_S) ? 1.0 / (8.0 * SPS_PI) : -3.0 / (4.0 * SPS_PI);
  k_reduce_parts<<<(int)std::min<long long>((n3 + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      n3, splits, ctx->d_part, scale, nullptr, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// FP32 far sum of kind kop (SPS_OP_S, SPS_OP_K or kOpKT): sources carry
// (Wsrc ? Wsrc : 1) * sig, the result is scaled by (Wtgt ? Wtgt : 1) * scale.
template <int KOP>
static int far32_run(sps_ctx* ctx, const double* sig, const double* Wsrc, const double* Wtgt, double scale,
                     double* out, int phase) {
  const long long NP = ctx->NP;
  const int P = ctx->T.P, N = ctx->N;
  const long long n3 = 3 * NP;
  {
    SpsPhase timer(ctx, SPS_PH_FAR_AUX);
    k_wsig32<<<(int)std::min<long long>((n3 + 255) / 256, 4096), 256, 0, ctx->stream>>>(NP, sig, Wsrc,
                                                                                       ctx->d_sig32);
    SPS_LAUNCHED(ctx);
  }
  // persistent grid over (target block, source split) items
  const int spc = std::max(1, kChunkNodes / P);
  const int narr = (KOP == kOpKT) ? 5 : 3;
  const size_t smem = (size_t)narr * spc * P * sizeof(float4) + (size_t)spc * 6 * sizeof(float);
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  cudaFuncAttributes fa;
  SPS_CUDA(ctx, cudaFuncGetAttributes(&fa, k_far32<KOP>));
  if (smem + fa.sharedSizeBytes > 48 * 1024)   // static + dynamic above the default limit
    SPS_CUDA(ctx, cudaFuncSetAttribute(k_far32<KOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_far32<KOP>, kT32, smem);
  const int resident = std::max(1, per_sm) * std::max(1, sms);
  const int n_tb = (int)((NP + kTPB32 - 1) / kTPB32);
  // enough items for the atomic queue to balance the load (>= 8 per block)
  int splits = (int)std::min<long long>(std::max(1, (8 * resident + n_tb - 1) / n_tb), (long long)N);
  splits = std::min(splits, 64);
  const int n_items = n_tb * splits;
  const int grid = std::min(n_items, resident);
  SPS_TRY(sps_grow(ctx, &ctx->d_part, ctx->cap_part, (size_t)splits * n3 + 1));
  int* d_work = reinterpret_cast<int*>(ctx->d_part + (size_t)splits * n3);
  SPS_CUDA(ctx, cudaMemsetAsync(d_work, 0, sizeof(int), ctx->stream));
  {
    SpsPhase timer(ctx, phase);
    k_far32<KOP><<<grid, kT32, smem, ctx->stream>>>(N, P, spc, n_tb, n_items, splits, ctx->d_rel32, ctx->d_N32,
                                                    ctx->d_sig32, ctx->d_chi, ctx->d_clo, ctx->d_near_ptr,
                                                    ctx->d_near_idx, d_work, ctx->d_part);
    SPS_LAUNCHED(ctx);
  }
  SpsPhase timer(ctx, SPS_PH_FAR_AUX);
  k_reduce_parts<<<(int)std::min<long long>((n3 + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      n3, splits, ctx->d_part, scale, Wtgt, out);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

int sps_launch_far(sps_ctx* ctx, int op, const double* sig, double* out, bool fp32) {
  const long long NP = ctx->NP;
  const int P = ctx->T.P, N = ctx->N;
  const int ph = (op == SPS_OP_S) ? SPS_PH_FAR_S : SPS_PH_FAR_K;
  if (!fp32 && sps_far_dw(ctx)) return far_dw_run(ctx, op, sig, out, SPS_PH_FAR_DW);
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
  if (op == SPS_OP_S) return far32_run<SPS_OP_S>(ctx, sig, ctx->d_W, nullptr, 1.0 / (8.0 * SPS_PI), out, ph);
  return far32_run<SPS_OP_K>(ctx, sig, ctx->d_W, nullptr, -3.0 / (4.0 * SPS_PI), out, ph);
}

// transposed far sums in FP32 (mixed-precision adjoint): S^T with the weights
// at the target, K^T = +3/(4 pi) w_t sum r (r.v)(r.n_s)/|r|^5
int sps_launch_far_T32(sps_ctx* ctx, int op, const double* v, double* out) {
  if (op == SPS_OP_S)
    return far32_run<SPS_OP_S>(ctx, v, nullptr, ctx->d_W, 1.0 / (8.0 * SPS_PI), out, SPS_PH_FAR_S);
  return far32_run<kOpKT>(ctx, v, nullptr, ctx->d_W, 3.0 / (4.0 * SPS_PI), out, SPS_PH_FAR_K);
}
