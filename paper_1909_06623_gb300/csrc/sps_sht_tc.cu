// Tensor-core VSH transforms of the mixed-precision path (Sec. 4.2, 5.4):
// the analysis coef_s = A sigma_s and the self synthesis out_s = Synth_op coef_s
// for every sphere s, as one batched product on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory).
//
//   Out[s][n] = sum_k X_s[k] B[n][k]
//
// One CTA of 128 threads takes 128 spheres and 64 matrix rows: the spheres are
// the MMA's M = 128 rows, the matrix rows its N = 64, the contraction K runs
// in chunks of 32, staged into one of two shared-memory buffers while the
// tensor core works on the other.  Both operands are split into three BF16 terms,
// x = h + m + l (h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)), and the
// six products hh, hm, mh, hl, lh, mm of a chunk accumulate in FP32 in tensor
// memory (the dropped products are 2^-24 relative), hh in one accumulator and
// the five smaller ones in another; the chunk results are summed per thread
// with Kahan compensation.  The tensor core's FP32 accumulation rounds less carefully
// than an FMA chain: one accumulator over the whole contraction lost about a
// decimal digit against the FP32 CUDA-core product; with 32-term chunks and
// the large and small products apart the transforms are as accurate as the
// FP32 product, and the mixed mobility solve more accurate (measured; 64-term
// chunks were 5% faster and gave back most of that gain).
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
#ifndef SPS_TC_KC
#define SPS_TC_KC 32
#endif
constexpr int kKC = SPS_TC_KC;             // K chunk (one FP32 accumulation in tensor memory)
#ifndef SPS_TC_NT
#define SPS_TC_NT 16
#endif
constexpr int kNT = SPS_TC_NT;             // N tile: one CTA per (128 spheres, kNT matrix rows)
static_assert(kNT == 16 || kNT == 32 || kNT == 64, "N tile of 16, 32 or 64 rows");
constexpr int kSBO = (kKC / 8) * 128;      // bytes between 8-row groups
constexpr int kABytes = kM * kKC * 2;      // one split of the A chunk
constexpr int kBBytes = kNT * kKC * 2;     // one split of the B chunk
constexpr int kStage = 3 * kABytes + 3 * kBBytes;   // one buffer: A and B, three splits each
constexpr int kAccBytes = 2 * kNT * kM * 4;   // per-thread Kahan sums (sum, compensation)
constexpr int kSmem = 2 * kStage + kAccBytes;   // double-buffered operands + sums
constexpr unsigned kSpin = 1u << 22;       // try_wait rounds before giving up
// tensor memory: two accumulator sets (chunks alternate), each with the hh
// products in one 64-column block and the five smaller products in the next,
// so the large terms never share an FP32 accumulator with the small ones
constexpr int kTmemCols = 4 * kNT;

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

// The input operand A (rows = spheres) split into three BF16 terms once per
// transform, in the layout the chunks are staged in: sphere block sb of 128,
// chunk kc, split sp -> kM * kKC elements at ((sb * nkc + kc) * 3 + sp) * kM * kKC,
// canonical K-major inside.  The FP64 -> FP32 conversion runs here, once per
// element, instead of in every CTA of every N tile.
template <int MODE>
__global__ void k_tc_split(int Ns, int P, int K, int nkc, const double* __restrict__ in,
                           uint16_t* __restrict__ Asp) {
  const long long NP = (long long)Ns * P;
  const int nsb = (Ns + kM - 1) / kM;
  const long long total = (long long)nsb * nkc * kM * (kKC / 8);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int it = (int)(q % (kM * (kKC / 8)));
    const long long bc = q / (kM * (kKC / 8));       // sb * nkc + kc
    const int kc = (int)(bc % nkc), sb = (int)(bc / nkc);
    const int r = it / (kKC / 8), k8 = (it % (kKC / 8)) * 8;
    const int s = sb * kM + r;
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
    unsigned char* base = reinterpret_cast<unsigned char*>(Asp + bc * 3 * (kM * kKC));
    const int off = tc_off(r, k8);
    *reinterpret_cast<uint4*>(base + off) = *reinterpret_cast<const uint4*>(vh);
    *reinterpret_cast<uint4*>(base + kABytes + off) = *reinterpret_cast<const uint4*>(vm);
    *reinterpret_cast<uint4*>(base + 2 * kABytes + off) = *reinterpret_cast<const uint4*>(vl);
  }
}

// stage K chunk kc: the pre-split A chunk of the CTA's spheres and the
// pre-split B chunk of this N tile, into one smem buffer (plain 16-byte copies)
__device__ __forceinline__ void stage_chunk(unsigned char* buf, const uint16_t* __restrict__ Achunk,
                                            const uint16_t* __restrict__ Bchunk, int nrows) {
  unsigned char* sA = buf;
  unsigned char* sB = buf + 3 * kABytes;
  const uint4* srcA = reinterpret_cast<const uint4*>(Achunk);
  for (int v = threadIdx.x; v < 3 * kABytes / 16; v += 128)
    *reinterpret_cast<uint4*>(sA + 16 * v) = srcA[v];
  const int bytes = nrows * kKC * 2;
  const uint4* src = reinterpret_cast<const uint4*>(Bchunk);
  for (int v = threadIdx.x; v < 3 * bytes / 16; v += 128) {
    const int sp = v / (bytes / 16), w = v % (bytes / 16);
    *reinterpret_cast<uint4*>(sB + sp * kBBytes + 16 * w) = src[v];
  }
  // generic-proxy smem writes -> visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// grid (sphere blocks of 128, N tiles of 64); 128 threads, thread t owns
// sphere s0 + t (tensor-memory lane t) and the tile's columns
template <int MODE>
__global__ void __launch_bounds__(128) k_sht_tc(int Ns, int P, int Nout, int K, int Kpad,
                                               const uint16_t* __restrict__ Bt,
                                               const uint16_t* __restrict__ Asp,
                                               double* __restrict__ out,
                                               const double* __restrict__ rad, int scale_by_radius,
                                               const double* __restrict__ sig, int half,
                                               int* __restrict__ flag) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int s0 = blockIdx.x * kM;
  const int t = blockIdx.y;
  const int nrows = tile_rows(Nout, t), n0 = t * kNT;
  const int nkc = Kpad / kKC;
  const long long NP = (long long)Ns * P;
  // tiles before t are full (kNT rows); chunk kc of tile t at tile base + kc * 3 * nrows * kKC
  const uint16_t* Btile = Bt + (size_t)t * 3 * kNT * Kpad;
  const uint16_t* Ablock = Asp + (size_t)blockIdx.x * nkc * 3 * (kM * kKC);
  const uint32_t bar0 = smem_u32(&bar[0]), bar1 = smem_u32(&bar[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  stage_chunk(smem, Ablock, Btile, nrows);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t id = idesc(nrows);
  // (A split, B split) of the six products kept; product 0 (hh) in its own accumulator
  auto issue = [&](int kc) {
    const int b = kc & 1;
    const uint32_t a0 = smem_u32(smem + b * kStage), b0 = a0 + 3 * kABytes;
    const uint32_t acc = tmem + (uint32_t)(b * 2 * kNT);
    const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
    for (int ks = 0; ks < kKC / 16; ++ks)
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const uint64_t da = sdesc(a0 + pa[q] * kABytes + ks * 256);
        const uint64_t db = sdesc(b0 + pb[q] * kBBytes + ks * 256);
        if (q == 0)
          mma_bf16(acc, da, db, id, ks > 0 ? 1 : 0);
        else
          mma_bf16(acc + kNT, da, db, id, (ks > 0 || q > 1) ? 1 : 0);
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b ? bar1 : bar0)
                 : "memory");
  };
  if (tid == 0) issue(0);

  // compensated FP32 sums of the chunk results, one per column of the tile,
  // in shared memory ([column][thread]: consecutive threads, consecutive words)
  float* sum = reinterpret_cast<float*>(smem + 2 * kStage);
  float* cmp = sum + kNT * kM;
  for (int c = 0; c < kNT; ++c) sum[c * kM + tid] = cmp[c * kM + tid] = 0.f;
  uint32_t par[2] = {0u, 0u};
  bool ok = true;
  for (int kc = 0; kc < nkc; ++kc) {
    if (kc + 1 < nkc) {
      // buffer (kc+1)&1 was read by chunk kc-1, whose completion was awaited
      stage_chunk(smem + ((kc + 1) & 1) * kStage, Ablock + (size_t)(kc + 1) * 3 * (kM * kKC),
                  Btile + (size_t)(kc + 1) * 3 * nrows * kKC, nrows);
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) issue(kc + 1);
    }
    const int b = kc & 1;
    ok = __syncthreads_and(bar_wait(b ? bar1 : bar0, par[b])) != 0;   // CTA-uniform outcome
    par[b] ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) break;
    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 2 * kNT);
    for (int c0 = 0; c0 < nrows; c0 += 16) {
      uint32_t v[16], w[16];
      tmem_ld16(ta + c0, v);
      tmem_ld16(ta + kNT + c0, w);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        // Kahan: sum += (hh part + small part)
        const int e = (c0 + u) * kM + tid;
        const float x = __uint_as_float(v[u]) + __uint_as_float(w[u]);
        const float sv = sum[e];
        const float y = x - cmp[e];
        const float z = sv + y;
        cmp[e] = (z - sv) - y;
        sum[e] = z;
      }
    }
    // the next issue into this accumulator set comes after a barrier preceded
    // by tcgen05.fence::before_thread_sync, so these reads complete first
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  if (ok) {
    const int s = s0 + tid;
    if (s < Ns) {
      const double sc = scale_by_radius ? rad[s] : 1.0;
      for (int c = 0; c < kNT; ++c) {
        const int n = n0 + c;
        if (c >= nrows || n >= Nout) continue;
        double val = ((double)sum[c * kM + tid] - (double)cmp[c * kM + tid]) * sc;
        if (MODE == MODE_ANALYSIS) {
          out[(long long)s * Nout + n] = val;
        } else {
          const int comp = n / P, kk = n - comp * P;
          const long long idx = comp * NP + (long long)s * P + kk;
          if (half) val += 0.5 * sig[idx];
          out[idx] = val;
        }
      }
    }
  } else {
    if (tid == 0) atomicOr(flag, 1);
    bar_wait(bar0, par[0]);   // one more bounded wait for MMAs in flight
    bar_wait(bar1, par[1]);
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
  const int nsb = (N + kM - 1) / kM, nkc = m.Kpad / kKC;
  SPS_TRY(sps_grow(ctx, &ctx->d_tcsplit, ctx->cap_tcsplit, (size_t)nsb * nkc * 3 * kM * kKC));
  const long long items = (long long)nsb * nkc * kM * (kKC / 8);
  const int sgrid = (int)std::min<long long>((items + 255) / 256, 8 * 152);
  if (mode == 0)
    k_tc_split<MODE_ANALYSIS><<<sgrid, 256, 0, ctx->stream>>>(N, P, m.C, nkc, in, ctx->d_tcsplit);
  else
    k_tc_split<MODE_SYNTH><<<sgrid, 256, 0, ctx->stream>>>(N, P, m.C, nkc, in, ctx->d_tcsplit);
  SPS_LAUNCHED(ctx);
  const dim3 grid(nsb, (m.R + kNT - 1) / kNT);
  if (mode == 0)
    k_sht_tc<MODE_ANALYSIS><<<grid, 128, kSmem, ctx->stream>>>(N, P, m.R, m.C, m.Kpad, m.d, ctx->d_tcsplit, out,
                                                               ctx->d_rad, scale_by_radius, sig, half,
                                                               ctx->d_tcflag);
  else
    k_sht_tc<MODE_SYNTH><<<grid, 128, kSmem, ctx->stream>>>(N, P, m.R, m.C, m.Kpad, m.d, ctx->d_tcsplit, out,
                                                            ctx->d_rad, scale_by_radius, sig, half,
                                                            ctx->d_tcflag);
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
