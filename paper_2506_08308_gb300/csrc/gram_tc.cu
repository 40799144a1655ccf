// Tall-skinny Gram G = A^T B of two pair blocks on the tensor cores
// (tcgen05.mma, accumulator in tensor memory).
//
// Every operand element x is split into three BF16 slices, x = x0 + x1 + x2
// (x0 the BF16 rounding of x, x1 of what x0 leaves, x2 of the rest), which
// holds x to about 2^-24.  Of the nine slice products the six whose weight
// reaches 2^-24 of the leading one are accumulated in FP32 by the MMA:
// x0 y0, x0 y1, x1 y0, x1 y1, x0 y2, x2 y0.  Each CTA sums a chunk of rows
// this way and writes its FP32 tile as FP64 partial sums; the chunks are
// summed in FP64.  The result has FP32 accuracy (a few 2^-24 of
// sum |a_k b_k|): it serves the Grams of the FP32 phase and the first pass
// of the two-pass Gram-Schmidt (whose second pass, in double-float, removes
// what the first one leaves).
//
// Layout of one pipeline stage in shared memory: for A (128 real columns)
// and B (NT real columns) three BF16 slice tiles of TBK = 32 rows each, in
// the K-major layout of the MMA without swizzle: core matrices of 8 columns
// x 8 rows (16 bytes per column), core matrix (k8, c8) at byte offset
// (k8 * (cols / 8) + c8) * 128.  One MMA step covers 16 rows (two core
// matrices along K, `lbo` bytes apart; 8-column groups `sbo` = 128 bytes
// apart).
#include <cuda_bf16.h>

#include <algorithm>

#include "blas.cuh"

namespace bdg {

namespace {

constexpr int TM = 128;          // A real columns per CTA (MMA M)
constexpr int TBK = 32;          // rows per pipeline stage (two MMA K steps of 16)
constexpr int TSTAGES = 2;       // stages in flight
constexpr int TTHREADS = 256;
constexpr int TNMAX = 160;       // widest B tile (real columns, multiple of 16)
constexpr int NSLICE = 3;
constexpr int A_SLICE_BYTES = TM * TBK * 2;
constexpr long long WAIT_LIMIT = 1LL << 22;  // polls of an MMA barrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor (no swizzle): start address, byte offset
// between the two core matrices along K, byte offset between 8-column
// groups, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  r -= __bfloat162float(b);
  c = __float2bfloat16_rn(r);
}

// FP64 x cut to FP32 by its bits (24 significant bits, truncated; below the
// FP32 normal range 0, above it infinity, NaN kept): no FP64 arithmetic,
// which runs at a small fraction of the FP32 rate on this part.
__device__ __forceinline__ float cut_to_float(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int ex = (int)((hi >> 20) & 0x7FFu);
  const unsigned mant = (unsigned)(b >> 29) & 0x7FFFFFu;
  if (ex == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (mant ? 0x400000u : 0u));
  const int e = ex - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}

__device__ __forceinline__ void split3(double x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  split3(cut_to_float(x), a, b, c);
}

// Rows r .. r+7 of complex column `col` (zero past r_end or past the
// block's columns) as the slices of real columns c (real parts) and c + 1
// (imaginary parts) of a tile of `tcols` columns: one 16-byte core-matrix
// row per slice and real column.
template <typename R>
__device__ __forceinline__ void stage_rows(const PairBlock<R>& X, int col, long long r, long long r_end, int c,
                                           int g, int tcols, uint8_t* base) {
  typedef typename CT<R>::T T;
  T v[8];
  const bool colok = col < X.cols;
  const T* src = X.p + (long long)(colok ? col : 0) * X.ld + r;
  if (colok && r + 8 <= r_end && ((uintptr_t)src & 15) == 0) {
    // whole group in range: 16-byte loads, all in flight together
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4 u[sizeof(T) / 2];
#pragma unroll
    for (int q = 0; q < (int)(sizeof(T) / 2); ++q) u[q] = __ldg(s4 + q);
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = reinterpret_cast<const T*>(u)[q];
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (colok && r + q < r_end) ? src[q] : mk((R)0, (R)0);
  }
  uint32_t w[2][NSLICE][4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    __nv_bfloat16 a0, b0, c0, a1, b1, c1;
    split3(v[q].x, a0, b0, c0);
    split3(v[q + 1].x, a1, b1, c1);
    w[0][0][q / 2] = pack2(a0, a1);
    w[0][1][q / 2] = pack2(b0, b1);
    w[0][2][q / 2] = pack2(c0, c1);
    split3(v[q].y, a0, b0, c0);
    split3(v[q + 1].y, a1, b1, c1);
    w[1][0][q / 2] = pack2(a0, a1);
    w[1][1][q / 2] = pack2(b0, b1);
    w[1][2][q / 2] = pack2(c0, c1);
  }
  const uint32_t slice_bytes = (uint32_t)tcols * TBK * 2;
  const uint32_t lbo = (uint32_t)(tcols / 8) * 128;
  // The eight threads of a quarter warp hold eight consecutive complex
  // columns of one K group: those with complex column % 8 >= 4 store the
  // imaginary row first, so that every 16-byte store of the quarter warp
  // lands in a different group of four banks.
  const int flip = (c >> 3) & 1;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int part = q ^ flip;
    const int cc = c + part;
    const uint32_t off = (uint32_t)g * lbo + (uint32_t)(cc / 8) * 128 + (uint32_t)(cc % 8) * 16;
#pragma unroll
    for (int s = 0; s < NSLICE; ++s) {
      const uint4 u0 = make_uint4(w[0][s][0], w[0][s][1], w[0][s][2], w[0][s][3]);
      const uint4 u1 = make_uint4(w[1][s][0], w[1][s][1], w[1][s][2], w[1][s][3]);
      *reinterpret_cast<uint4*>(base + s * slice_bytes + off) = part ? u1 : u0;
    }
  }
}

// Partial Gram of one row chunk: part[chunk][i][j] for real columns
// i < 2 A.cols (128 per CTA along x), j < 2 B.cols <= NT.  A wait that runs
// out writes NaN into the tile (the caller sees a NaN Gram).
template <typename R>
__global__ void __launch_bounds__(TTHREADS, 2)
    k_gram_tc(PairBlock<R> A, PairBlock<R> B, int NT, long long crows, double* __restrict__ part) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_slice = (uint32_t)NT * TBK * 2;
  const uint32_t stage_bytes = NSLICE * (A_SLICE_BYTES + b_slice);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + TSTAGES * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + TSTAGES);
  const uint32_t ncols = NT <= 32 ? 32u : NT <= 64 ? 64u : NT <= 128 ? 128u : 256u;
  const int i0 = blockIdx.x * TM;
  const long long r_begin = (long long)blockIdx.z * crows;
  const long long r_end = min(A.n, r_begin + crows);
  const int P2 = 2 * A.cols, Q2 = 2 * B.cols;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < TSTAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nsteps = r_end > r_begin ? (int)((r_end - r_begin + TBK - 1) / TBK) : 0;
  bool lost = false;
  for (int step = 0; step < nsteps; ++step) {
    const int st = step % TSTAGES;
    uint8_t* sa = smem + st * stage_bytes;
    uint8_t* sb = sa + NSLICE * A_SLICE_BYTES;
    // the MMAs that read this stage (committed TSTAGES steps ago) are done
    if (step >= TSTAGES && !mbar_wait(smem_u32(&mbar[st]), (uint32_t)((step / TSTAGES - 1) & 1))) lost = true;
    const long long r0 = r_begin + (long long)step * TBK;
    // A: 64 complex columns x 4 groups of 8 rows, one group per thread;
    // task t -> column (t & 7) + 8 (t >> 5), group (t >> 3) & 3: a quarter
    // warp covers eight consecutive columns of one group
    {
      const int c = (tid & 7) | ((tid >> 5) << 3), g = (tid >> 3) & 3;
      stage_rows<R>(A, i0 / 2 + c, r0 + 8 * g, r_end, 2 * c, g, TM, sa);
    }
    for (int t = tid; t < (NT / 2) * 4; t += TTHREADS) {
      const int c = (t & 7) | ((t >> 5) << 3), g = (t >> 3) & 3;
      stage_rows<R>(B, c, r0 + 8 * g, r_end, 2 * c, g, NT, sb);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = idesc_bf16(TM, NT);
      const uint32_t lbo_a = (TM / 8) * 128, lbo_b = (uint32_t)(NT / 8) * 128;
      // slice pairs (A slice, B slice) whose weight reaches 2^-24 of the leading one
      const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
      for (int p = 0; p < 6; ++p)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint64_t ad = sdesc(smem_u32(sa + pa[p] * A_SLICE_BYTES + 2 * kk * lbo_a), lbo_a, 128);
          const uint64_t bd = sdesc(smem_u32(sb + pb[p] * b_slice + 2 * kk * lbo_b), lbo_b, 128);
          const uint32_t acc = (step > 0 || p > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[st]))
                   : "memory");
    }
  }
  if (nsteps > 0) {
    const int last = nsteps - 1;
    if (!mbar_wait(smem_u32(&mbar[last % TSTAGES]), (uint32_t)((last / TSTAGES) & 1))) lost = true;
  }
  lost = __syncthreads_or(lost) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int quarter = warp & 3;  // a warp reads TMEM lanes 32 quarter .. 32 quarter + 31
  const int i = i0 + 32 * quarter + lane;
  double* out = part + (long long)blockIdx.z * P2 * Q2;
  for (int jc = (warp >> 2) * 16; jc < NT; jc += 32) {
    uint32_t v[16];
    if (nsteps > 0) {
      const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)jc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = 0u;
    }
    if (i < P2) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = jc + q;
        if (j < Q2) out[(long long)i * Q2 + j] = lost ? (double)NAN : (double)__uint_as_float(v[q]);
      }
    }
  }
  if (lost && nsteps > 0) {
    // the MMAs may still run: wait (bounded) for the last commit before freeing their accumulator
    const int last = nsteps - 1;
    mbar_wait(smem_u32(&mbar[last % TSTAGES]), (uint32_t)((last / TSTAGES) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// G[e] = sum over chunks, in a fixed order: thread (x, y) of a 32 x 8 block
// sums chunks y, y + 8, ... of output e (independent loads in flight), then
// the eight sums are added in order of y.
__global__ void __launch_bounds__(256) k_gram_tc_reduce(const double* __restrict__ part, int nchunks, int nout,
                                                        double* __restrict__ G) {
  __shared__ double t[8][33];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + x;
  double s = 0.0;
  if (e < nout)
#pragma unroll 4
    for (int c = y; c < nchunks; c += 8) s += part[(long long)c * nout + e];
  t[y][x] = s;
  __syncthreads();
  if (y == 0 && e < nout) {
    double g = t[0][x];
#pragma unroll
    for (int q = 1; q < 8; ++q) g += t[q][x];
    G[e] = g;
  }
}

size_t tc_smem_bytes(int NT) {
  return (size_t)TSTAGES * NSLICE * (A_SLICE_BYTES + (size_t)NT * TBK * 2) + 8 * TSTAGES + 16;
}

}  // namespace

bool gram_tc_supported(int P, int Q) { return P > 0 && Q > 0 && 2 * Q <= TNMAX; }

template <typename R>
cudaError_t gram_pairs_tc(const PairBlock<R>& A, const PairBlock<R>& B, double* G_dev, void* ws,
                          size_t ws_bytes, cudaStream_t s) {
  if (A.n != B.n) return cudaErrorInvalidValue;
  const int P2 = 2 * A.cols, Q2 = 2 * B.cols;
  if (P2 == 0 || Q2 == 0) return cudaSuccess;
  if (!gram_tc_supported(A.cols, B.cols)) return cudaErrorNotSupported;
  if (A.n == 0) return cudaMemsetAsync(G_dev, 0, sizeof(double) * P2 * Q2, s);
  const int NT = (Q2 + 15) / 16 * 16;
  const int mtiles = (P2 + TM - 1) / TM;
  const size_t per_chunk = sizeof(double) * (size_t)P2 * Q2;
  const long long cap = (long long)(ws_bytes / per_chunk);
  if (cap < 1) return cudaErrorInvalidValue;
  // about two CTAs per SM (each holds two stages and 32 ... 256 TMEM columns)
  long long nch = std::min<long long>((2 * 152 + mtiles - 1) / mtiles, cap);
  nch = std::min<long long>(nch, (A.n + TBK - 1) / TBK);
  const long long crows = ((A.n + nch - 1) / nch + TBK - 1) / TBK * TBK;
  nch = (A.n + crows - 1) / crows;
  const size_t smem = tc_smem_bytes(NT);
  cudaError_t e = allow_dynamic_smem((const void*)k_gram_tc<R>, smem);
  if (e != cudaSuccess) return e;
  k_gram_tc<R><<<dim3((unsigned)mtiles, 1, (unsigned)nch), TTHREADS, smem, s>>>(A, B, NT, crows, (double*)ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nout = P2 * Q2;
  k_gram_tc_reduce<<<(nout + 31) / 32, 256, 0, s>>>((const double*)ws, (int)nch, nout, G_dev);
  return cudaGetLastError();
}

template cudaError_t gram_pairs_tc<float>(const PairBlock<float>&, const PairBlock<float>&, double*, void*, size_t,
                                          cudaStream_t);
template cudaError_t gram_pairs_tc<double>(const PairBlock<double>&, const PairBlock<double>&, double*, void*,
                                           size_t, cudaStream_t);

}  // namespace bdg
