// Tensor-core VSH transforms of the mixed-precision path (Sec. 4.2, 5.4):
// the analysis coef_s = A sigma_s and the self synthesis out_s = Synth_op coef_s
// for every sphere s, as one batched product on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory).
//
//   Out[s][n] = sum_k X_s[k] B[n][k]
//
// One CTA of 128 threads takes 128 spheres: the spheres are the MMA's M = 128
// rows, the matrix rows its N (tiles of at most 256), the contraction K runs
// in chunks of 32.  Both operands are split into three BF16 terms,
// x = h + m + l (h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)), and the
// six products hh, hm, mh, hl, lh, mm of a chunk accumulate in FP32 in tensor
// memory (the dropped products are 2^-24 relative), hh in one accumulator and
// the five smaller ones in another; the accumulators and the chunk sums are
// then added in FP64.  The tensor core's FP32 accumulation rounds less carefully
// than an FMA chain: one accumulator over the whole contraction lost about a
// decimal digit against the FP32 CUDA-core product; with 32-term chunks and
// the large and small products apart the transforms are as accurate as the
// FP32 product, and the mixed mobility solve more accurate (measured).
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8 x 16-byte core matrices, adjacent along K 128 bytes apart (leading byte
// offset), adjacent along M / N 512 bytes apart (stride byte offset: the 4
// core matrices of a 32-wide K chunk).  The constant matrix B is stored in global
// memory already split and laid out chunk by chunk, so staging it is a copy.
// One thread issues the MMAs; tcgen05.commit signals an mbarrier that every
// thread waits on with a bounded spin (on timeout the kernel records the
// failure in *flag, releases its tensor memory and returns).
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "sps_internal.cuh"

namespace {

constexpr int kM = 128;                    // spheres per CTA (MMA M)
constexpr int kKC = 32;                    // K chunk (one FP32 accumulation in tensor memory)
constexpr int kNT = 256;                   // widest N tile
constexpr int kSBO = (kKC / 8) * 128;      // bytes between 8-row groups
constexpr int kABytes = kM * kKC * 2;      // one split of the A chunk
constexpr int kBBytes = kNT * kKC * 2;     // one split of the B chunk (widest tile)
constexpr int kSmem = 3 * kABytes + 3 * kBBytes;
constexpr unsigned kSpin = 1u << 22;       // try_wait rounds before giving up
// the hh products accumulate in columns [0, 256), the five smaller products in
// [256, 512): the large terms never share an FP32 accumulator with the small ones
constexpr int kTmemCols = 2 * kNT;

enum { MODE_ANALYSIS = 0, MODE_SYNTH = 1 };

// byte offset of element (row r, k) of a K-major chunk
__host__ __device__ __forceinline__ int tc_off(int r, int k) {
  return (r >> 3) * kSBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__host__ __device__ __forceinline__ int tile_rows(int Nout, int t) {
  const int n = Nout - t * kNT;
  const int w = n < kNT ? n : kNT;
  return (w + 15) & ~15;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(kSBO >> 4) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta));
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < kSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

template <int MODE>
__global__ void __launch_bounds__(128, 1) k_sht_tc(int Ns, int P, int Nout, int K, int Kpad,
                                                  const uint16_t* __restrict__ Bt,
                                                  const double* __restrict__ in,
                                                  double* __restrict__ out,
                                                  const double* __restrict__ rad, int scale_by_radius,
                                                  const double* __restrict__ sig, int half,
                                                  int* __restrict__ flag) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  unsigned char* sA = smem;                  // 3 splits x kABytes
  unsigned char* sB = smem + 3 * kABytes;    // 3 splits x kBBytes
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = blockIdx.x * kM;
  const long long NP = (long long)Ns * P;
  const uint32_t bar_a = smem_u32(&bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  uint32_t parity = 0;
  bool ok = true;

  const int ntiles = (Nout + kNT - 1) / kNT;
  const int nkc = Kpad / kKC;
  size_t tbase = 0;                           // element offset of tile t in Bt
  for (int t = 0; t < ntiles && ok; ++t) {
    const int nrows = tile_rows(Nout, t);
    const int n0 = t * kNT;
    const uint32_t id = idesc(nrows);
    for (int kc = 0; kc < nkc && ok; ++kc) {
      // ---- stage A: rows = spheres, 8 consecutive k per item (one core-matrix row)
      for (int it = tid; it < kM * (kKC / 8); it += 128) {
        const int r = it / (kKC / 8), k8 = (it % (kKC / 8)) * 8;
        const int s = s0 + r;
        __align__(16) __nv_bfloat16 vh[8], vm[8], vl[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = kc * kKC + k8 + u;
          float x = 0.f;
          if (s < Ns && k < K) {
            if (MODE == MODE_ANALYSIS) {
              const int comp = k / P, kk = k - comp * P;
              x = (float)in[comp * NP + (long long)s * P + kk];
            } else {
              x = (float)in[(long long)s * K + k];
            }
          }
          split3(x, vh[u], vm[u], vl[u]);
        }
        const int off = tc_off(r, k8);
        *reinterpret_cast<uint4*>(sA + off) = *reinterpret_cast<const uint4*>(vh);
        *reinterpret_cast<uint4*>(sA + kABytes + off) = *reinterpret_cast<const uint4*>(vm);
        *reinterpret_cast<uint4*>(sA + 2 * kABytes + off) = *reinterpret_cast<const uint4*>(vl);
      }
      // ---- stage B: the pre-split chunk (3 x nrows x 64 BF16, already laid out)
      {
        const int bytes = nrows * kKC * 2;
        const uint4* src = reinterpret_cast<const uint4*>(Bt + tbase + (size_t)kc * 3 * nrows * kKC);
        for (int v = tid; v < 3 * bytes / 16; v += 128) {
          const int sp = v / (bytes / 16), w = v % (bytes / 16);
          *reinterpret_cast<uint4*>(sB + sp * kBBytes + 16 * w) = src[v];
        }
      }
      // generic-proxy smem writes -> visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        // (A split, B split) of the six products kept
        const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
        for (int ks = 0; ks < kKC / 16; ++ks)
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const uint64_t da = sdesc(a0 + pa[q] * kABytes + ks * 256);
            const uint64_t db = sdesc(b0 + pb[q] * kBBytes + ks * 256);
            if (q == 0)
              mma_bf16(tmem, da, db, id, ks > 0 ? 1 : 0);
            else
              mma_bf16(tmem + kNT, da, db, id, (ks > 0 || q > 1) ? 1 : 0);
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                     : "memory");
      }
      ok = __syncthreads_and(bar_wait(bar_a, parity)) != 0;   // CTA-uniform outcome
      parity ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (!ok) break;
      // ---- the chunk's partial sums (warp w reads tensor-memory lanes 32w..),
      // added in FP64 to the previous chunks'; scaling on the last chunk
      const int r = warp * 32 + lane;
      const int s = s0 + r;
      const bool first = (kc == 0), last = (kc == nkc - 1);
      for (int c0 = 0; c0 < nrows; c0 += 16) {
        uint32_t v[16], w[16];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        tmem_ld16(ta, v);
        tmem_ld16(ta + kNT, w);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (s < Ns) {
          const double sc = scale_by_radius ? rad[s] : 1.0;
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int n = n0 + c0 + u;
            if (n >= Nout) continue;
            long long idx;
            if (MODE == MODE_ANALYSIS) {
              idx = (long long)s * Nout + n;
            } else {
              const int comp = n / P, kk = n - comp * P;
              idx = comp * NP + (long long)s * P + kk;
            }
            double acc = (double)__uint_as_float(v[u]) + (double)__uint_as_float(w[u]);
            if (!first) acc += out[idx];
            if (last) {
              acc *= sc;
              if (MODE == MODE_SYNTH && half) acc += 0.5 * sig[idx];
            }
            out[idx] = acc;
          }
        }
      }
    }
    tbase += (size_t)3 * nrows * Kpad;
    // staging for the next chunk or tile is preceded by a barrier with
    // tcgen05.fence::before_thread_sync, so these tensor-memory reads complete
    // before the next MMAs overwrite the accumulator
  }
  if (!ok) {
    if (tid == 0) atomicOr(flag, 1);
    bar_wait(bar_a, parity);   // one more bounded wait for the MMAs in flight
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

uint16_t bf16_bits(float x) {
  // round to nearest even (finite inputs)
  uint32_t u;
  std::memcpy(&u, &x, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}
float bf16_val(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}

}  // namespace

// Splits the R x C matrix M (row n = output, column k = contraction) into the
// tile / chunk / split layout read by k_sht_tc and uploads it.
int sps_sht_tc_upload(sps_ctx* ctx, sps_ctx::TcMat& out, const std::vector<double>& M, int R, int C) {
  const int Kpad = (C + kKC - 1) / kKC * kKC;
  const int ntiles = (R + kNT - 1) / kNT;
  size_t total = 0;
  for (int t = 0; t < ntiles; ++t) total += (size_t)3 * tile_rows(R, t) * Kpad;
  std::vector<uint16_t> h(total, 0);
  size_t tbase = 0;
  for (int t = 0; t < ntiles; ++t) {
    const int nrows = tile_rows(R, t);
    for (int kc = 0; kc < Kpad / kKC; ++kc) {
      const size_t cbase = tbase + (size_t)kc * 3 * nrows * kKC;
      for (int r = 0; r < nrows; ++r)
        for (int k = 0; k < kKC; ++k) {
          const int n = t * kNT + r, c = kc * kKC + k;
          const float x = (n < R && c < C) ? (float)M[(size_t)n * C + c] : 0.f;
          const uint16_t hb = bf16_bits(x);
          const float r1 = x - bf16_val(hb);
          const uint16_t mb = bf16_bits(r1);
          const uint16_t lb = bf16_bits(r1 - bf16_val(mb));
          const size_t e = (size_t)tc_off(r, k) / 2;
          h[cbase + e] = hb;
          h[cbase + (size_t)nrows * kKC + e] = mb;
          h[cbase + 2 * (size_t)nrows * kKC + e] = lb;
        }
    }
    tbase += (size_t)3 * nrows * Kpad;
  }
  SPS_CUDA(ctx, cudaMalloc((void**)&out.d, sizeof(uint16_t) * total));
  SPS_CUDA(ctx, cudaMemcpy(out.d, h.data(), sizeof(uint16_t) * total, cudaMemcpyHostToDevice));
  out.R = R;
  out.C = C;
  out.Kpad = Kpad;
  return SPS_OK;
}

// mode 0: analysis (in = density planes, out = N x R coefficient rows);
// mode 1: synthesis (in = N x C coefficient rows, out = field planes, times the
// radius if scale_by_radius, plus sig / 2 if half)
int sps_launch_sht_tc(sps_ctx* ctx, const sps_ctx::TcMat& m, int mode, const double* in, double* out,
                      int scale_by_radius, const double* sig, int half) {
  const int N = ctx->N, P = ctx->T.P;
  if (!ctx->d_tcflag) {
    size_t c = 0;
    SPS_TRY(sps_grow(ctx, &ctx->d_tcflag, c, 1));
    SPS_CUDA(ctx, cudaMemsetAsync(ctx->d_tcflag, 0, sizeof(int), ctx->stream));
  }
  static bool attr = false;
  if (!attr) {
    SPS_CUDA(ctx, cudaFuncSetAttribute(k_sht_tc<MODE_ANALYSIS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    SPS_CUDA(ctx, cudaFuncSetAttribute(k_sht_tc<MODE_SYNTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    attr = true;
  }
  const int grid = (N + kM - 1) / kM;
  if (mode == 0)
    k_sht_tc<MODE_ANALYSIS><<<grid, 128, kSmem, ctx->stream>>>(N, P, m.R, m.C, m.Kpad, m.d, in, out, ctx->d_rad,
                                                               scale_by_radius, sig, half, ctx->d_tcflag);
  else
    k_sht_tc<MODE_SYNTH><<<grid, 128, kSmem, ctx->stream>>>(N, P, m.R, m.C, m.Kpad, m.d, in, out, ctx->d_rad,
                                                            scale_by_radius, sig, half, ctx->d_tcflag);
  SPS_LAUNCHED(ctx);
  return SPS_OK;
}

// 0 if every tensor-core transform so far completed (reads a device flag)
int sps_sht_tc_status(sps_ctx* ctx) {
  if (!ctx->d_tcflag) return SPS_OK;
  int f = 0;
  SPS_CUDA(ctx, cudaMemcpyAsync(&f, ctx->d_tcflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (f) return sps_fail(ctx, SPS_ERR_CUDA, "tensor-core VSH transform timed out");
  return SPS_OK;
}
