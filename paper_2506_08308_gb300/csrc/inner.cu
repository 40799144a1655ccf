// Inner PCG of the subspace iteration's search directions (see inner.cuh).
#include <cstdlib>
#include <string>

#include "blas.cuh"
#include "inner.cuh"
#include "kdiag.cuh"
#include "plan.cuh"

namespace bdg {

namespace {

constexpr int NT = 256;
constexpr int NQ_MAX = 8;   // reduced quantities per complex column: 4 CG sums, or 4 Z columns x (re, im)
static_assert(NQ_MAX <= NT / 32, "sum_partials gives every quantity a warp");

// Block-wide sum of nq per-thread values in FP64, deterministic (fixed
// shuffle tree, then warps in order); the result lands in out[0..nq) of
// shared memory, valid after the trailing barrier.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], int nq, double* red /* [NT/32][NQ] */, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
    for (int q = 0; q < nq; ++q) red[warp * NQ + q] = v[q];
  __syncthreads();
  if (threadIdx.x < nq) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w * NQ + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// out[q] = sum over the nchunk partials of quantity q of complex column
// `pair` (layout part[(pair * nchunk + chunk) * nq + q]), in a fixed order:
// warp q, lane l sums chunks l, l + 32, ..., then a shuffle tree (the nq <=
// NT / 32 quantities in parallel, one warp each).
__device__ __forceinline__ void sum_partials(const double* __restrict__ part, int pair, int nchunk, int nq,
                                             double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < nq) {
    double t = 0.0;
    for (int c = lane; c < nchunk; c += 32) t += part[((long long)pair * nchunk + c) * nq + warp];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) out[warp] = t;
  }
  __syncthreads();
}

// Partial sums a.x b.x and a.y b.y over the f rows [0, n3) and the g rows
// [n3, 2 n3) of every complex column: q = (f re, f im, g re, g im).
template <typename R>
__global__ void __launch_bounds__(NT) k_pair_dots(const typename CT<R>::T* __restrict__ a,
                                                  const typename CT<R>::T* __restrict__ b, long long n3,
                                                  int nchunk, double* __restrict__ part) {
  typedef typename CT<R>::T T;
  __shared__ double red[NT / 32 * 4];
  __shared__ double out[4];
  const int pair = blockIdx.y, chunk = blockIdx.x;
  const long long vlen = 2 * n3, len = (vlen + nchunk - 1) / nchunk;
  const long long r0 = chunk * len, r1 = min(vlen, r0 + len);
  const T* ap = a + (long long)pair * vlen;
  const T* bp = b + (long long)pair * vlen;
  R s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (long long r = r0 + threadIdx.x; r < min(r1, n3); r += NT) {
    const T x = ap[r], y = bp[r];
    s0 = fma(x.x, y.x, s0);
    s1 = fma(x.y, y.y, s1);
  }
  for (long long r = max(r0, n3) + threadIdx.x; r < r1; r += NT) {
    const T x = ap[r], y = bp[r];
    s2 = fma(x.x, y.x, s2);
    s3 = fma(x.y, y.y, s3);
  }
  double v[4] = {(double)s0, (double)s1, (double)s2, (double)s3};
  block_sum<4>(v, 4, red, out);
  if (threadIdx.x < 4) part[((long long)pair * nchunk + chunk) * 4 + threadIdx.x] = out[threadIdx.x];
}

// x = alpha p (first step) or x + alpha p;  r -= alpha q, with
// alpha = rz / (p, q) per recurrence (0 where (p, q) <= 0: a direction
// without curvature, e.g. a zero column, adds nothing).
template <typename R>
__global__ void __launch_bounds__(NT) k_cg_xr(typename CT<R>::T* __restrict__ x, typename CT<R>::T* __restrict__ r,
                                              const typename CT<R>::T* __restrict__ p,
                                              const typename CT<R>::T* __restrict__ q, long long n3, int nchunk,
                                              const double* __restrict__ part, const double* __restrict__ rz,
                                              int first) {
  typedef typename CT<R>::T T;
  __shared__ double pq[4];
  __shared__ R al[4];
  const int pair = blockIdx.y;
  sum_partials(part, pair, nchunk, 4, pq);
  if (threadIdx.x < 4) {
    const double d = pq[threadIdx.x];
    al[threadIdx.x] = (R)(d > 0.0 ? rz[pair * 4 + threadIdx.x] / d : 0.0);
  }
  __syncthreads();
  const long long vlen = 2 * n3, off = (long long)pair * vlen;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < vlen; e += (long long)gridDim.x * NT) {
    const int h = e < n3 ? 0 : 2;
    const R ax = al[h], ay = al[h + 1];
    const T pv = p[off + e], qv = q[off + e];
    T xv = first ? mk((R)0, (R)0) : x[off + e];
    T rv = r[off + e];
    xv = mk(fma(ax, pv.x, xv.x), fma(ay, pv.y, xv.y));
    rv = mk(fma(-ax, qv.x, rv.x), fma(-ay, qv.y, rv.y));
    x[off + e] = xv;
    r[off + e] = rv;
  }
}

// p = z (first) or z + beta p with beta = (r, z)_new / (r, z)_old; the new
// (r, z) is stored in rz_out by the first CTA of each column.
template <typename R>
__global__ void __launch_bounds__(NT) k_cg_p(typename CT<R>::T* __restrict__ p, const typename CT<R>::T* __restrict__ z,
                                             long long n3, int nchunk, const double* __restrict__ part,
                                             const double* __restrict__ rz_in, double* __restrict__ rz_out,
                                             int first) {
  typedef typename CT<R>::T T;
  __shared__ double rzn[4];
  __shared__ R be[4];
  const int pair = blockIdx.y;
  sum_partials(part, pair, nchunk, 4, rzn);
  if (threadIdx.x < 4) {
    const double o = first ? 0.0 : rz_in[pair * 4 + threadIdx.x];
    be[threadIdx.x] = (R)(o != 0.0 ? rzn[threadIdx.x] / o : 0.0);
    if (blockIdx.x == 0) rz_out[pair * 4 + threadIdx.x] = rzn[threadIdx.x];
  }
  __syncthreads();
  const long long vlen = 2 * n3, off = (long long)pair * vlen;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < vlen; e += (long long)gridDim.x * NT) {
    const int h = e < n3 ? 0 : 2;
    const T zv = z[off + e];
    if (first) {
      p[off + e] = zv;
    } else {
      const T pv = p[off + e];
      p[off + e] = mk(fma(be[h], pv.x, zv.x), fma(be[h + 1], pv.y, zv.y));
    }
  }
}

// Coefficients of the swapped deflation: f rows against the nzg <= 1 columns
// of Z_g, g rows against the nzf <= 3 columns of Z_f (real orthonormal
// columns stored as complex with zero imaginary parts, column stride n3).
// Quantities per complex column: slots (0, 1) = (re, im) for the Z_g column,
// slots 2 + 2 c + (re, im) for Z_f column c.
template <typename R>
__global__ void __launch_bounds__(NT) k_zdots(const typename CT<R>::T* __restrict__ v,
                                              const typename CT<R>::T* __restrict__ zf, int nzf,
                                              const typename CT<R>::T* __restrict__ zg, int nzg, long long n3,
                                              int nchunk, double* __restrict__ part) {
  typedef typename CT<R>::T T;
  __shared__ double red[NT / 32 * NQ_MAX];
  __shared__ double out[NQ_MAX];
  const int pair = blockIdx.y, chunk = blockIdx.x;
  const long long vlen = 2 * n3, len = (vlen + nchunk - 1) / nchunk;
  const long long r0 = chunk * len, r1 = min(vlen, r0 + len);
  const T* vp = v + (long long)pair * vlen;
  R s[NQ_MAX];
#pragma unroll
  for (int q = 0; q < NQ_MAX; ++q) s[q] = 0;
  if (nzg > 0)
    for (long long r = r0 + threadIdx.x; r < min(r1, n3); r += NT) {
      const T x = vp[r];
      const R zv = zg[r].x;
      s[0] = fma(zv, x.x, s[0]);
      s[1] = fma(zv, x.y, s[1]);
    }
  for (long long r = max(r0, n3) + threadIdx.x; r < r1; r += NT) {
    const T x = vp[r];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < nzf) {
        const R zv = zf[c * n3 + (r - n3)].x;
        s[2 + 2 * c] = fma(zv, x.x, s[2 + 2 * c]);
        s[3 + 2 * c] = fma(zv, x.y, s[3 + 2 * c]);
      }
  }
  double d[NQ_MAX];
#pragma unroll
  for (int q = 0; q < NQ_MAX; ++q) d[q] = (double)s[q];
  block_sum<NQ_MAX>(d, NQ_MAX, red, out);
  if (threadIdx.x < NQ_MAX) part[((long long)pair * nchunk + chunk) * NQ_MAX + threadIdx.x] = out[threadIdx.x];
}

// v -= Z c with the coefficients of k_zdots (summed here in a fixed order)
template <typename R>
__global__ void __launch_bounds__(NT) k_zsub(typename CT<R>::T* __restrict__ v, const typename CT<R>::T* __restrict__ zf,
                                             int nzf, const typename CT<R>::T* __restrict__ zg, int nzg, long long n3,
                                             int nchunk, const double* __restrict__ part) {
  typedef typename CT<R>::T T;
  __shared__ double cf[NQ_MAX];
  const int pair = blockIdx.y;
  sum_partials(part, pair, nchunk, NQ_MAX, cf);
  const long long vlen = 2 * n3, off = (long long)pair * vlen;
  const long long stride = (long long)gridDim.x * NT;
  // ZB elements per thread and batch, all loads of a batch issued before its
  // stores (a load after a store to v could not be moved ahead of it)
  constexpr int ZB = 4;
  for (long long e0 = (long long)blockIdx.x * NT + threadIdx.x; e0 < vlen; e0 += ZB * stride) {
    T x[ZB];
    R z[ZB][3];
#pragma unroll
    for (int b = 0; b < ZB; ++b) {
      const long long e = e0 + b * stride;
      x[b] = mk((R)0, (R)0);
      z[b][0] = z[b][1] = z[b][2] = (R)0;
      if (e >= vlen) continue;
      x[b] = v[off + e];
      if (e < n3) {
        if (nzg > 0) z[b][0] = zg[e].x;
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c < nzf) z[b][c] = zf[c * n3 + (e - n3)].x;
      }
    }
#pragma unroll
    for (int b = 0; b < ZB; ++b) {
      const long long e = e0 + b * stride;
      if (e >= vlen) continue;
      T y = x[b];
      if (e < n3) {
        if (nzg > 0) y = mk(fma(-z[b][0], (R)cf[0], y.x), fma(-z[b][0], (R)cf[1], y.y));
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c < nzf) y = mk(fma(-z[b][c], (R)cf[2 + 2 * c], y.x), fma(-z[b][c], (R)cf[3 + 2 * c], y.y));
      }
      v[off + e] = y;
    }
  }
}

unsigned row_blocks(long long vlen) {
  long long b = (vlen + NT * 4 - 1) / (NT * 4);
  if (b > 1024) b = 1024;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

template <typename RI>
bdg_status InnerPCG<RI>::dots(const T* a, const T* b, int pairs, cudaStream_t s) {
  k_pair_dots<RI><<<dim3(nchunk_, pairs), NT, 0, s>>>(a, b, 3 * np_, nchunk_, part_);
  BDG_CUDA_TRY(plan_, cudaGetLastError());
  return BDG_OK;
}

template <typename RI>
bdg_status InnerPCG<RI>::deflate_swapped(T* v, int pairs, cudaStream_t s) {
  const int nzf = plan_->nzf, nzg = plan_->nzg;
  if (nzf + nzg == 0) return BDG_OK;
  if (nzf > 3 || nzg > 1) return fail(plan_, BDG_ERR_UNSUPPORTED, "inner solver: deflation space too large");
  k_zdots<RI><<<dim3(nchunk_, pairs), NT, 0, s>>>(v, zf_, nzf, zg_, nzg, 3 * np_, nchunk_, zpart_);
  BDG_CUDA_TRY(plan_, cudaGetLastError());
  k_zsub<RI><<<dim3(row_blocks(vlen_), pairs), NT, 0, s>>>(v, zf_, nzf, zg_, nzg, 3 * np_, nchunk_, zpart_);
  BDG_CUDA_TRY(plan_, cudaGetLastError());
  return BDG_OK;
}

template <typename RI>
bdg_status InnerPCG<RI>::precondition(const T* x, T* y, int pairs, double sigma, cudaStream_t s) {
  KdArgs<RI> g;
  g.grid = &plan_->grid;
  g.x = x;
  g.y = y;
  g.nplanes = 6LL * pairs;
  for (int a = 0; a < 3; ++a)
    g.tw[a] = (const T*)(sizeof(RI) == 8 ? (const void*)plan_->tw64[a] : (const void*)plan_->tw32[a]);
  g.shift = sigma;
  g.scale = 0.5;
  g.stream = s;
  BDG_CUDA_TRY(plan_, kdiag_launch<RI>(g));
  return BDG_OK;
}

template <typename RI>
void InnerPCG<RI>::release_graphs() {
  for (auto& g : graphs_)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  graphs_.clear();
  if (cap_) cudaStreamDestroy(cap_);
  cap_ = nullptr;
}

template <typename RI>
template <typename R>
bdg_status InnerPCG<RI>::run(const typename CT<R>::T* Rin, typename CT<R>::T* D, int pairs, int steps,
                             double sigma, cudaStream_t s) {
  if (pairs <= 0) return BDG_OK;
  if (pairs > max_pairs_) return fail(plan_, BDG_ERR_INVALID, "inner solver: block wider than its buffers");
  // products issued per call: one per step on the pairs, both halves
  if (sizeof(RI) == 8) plan_->stats.applies_fp64 += 2 * pairs * steps;
  else plan_->stats.applies_fp32 += 2 * pairs * steps;
  // graphs pay where launches are many and kernels short enough for the
  // host's launch time to matter: grids of 2^16 points and more
  const bool graphs_env = !getenv("BDG_INNER_GRAPHS") || atoi(getenv("BDG_INNER_GRAPHS")) != 0;
  if (!graphs_env || !use_graphs_ || np_ < (1LL << 16)) return run_direct<R>(Rin, D, pairs, steps, sigma, s);
  Graph* g = nullptr;
  for (auto& e : graphs_)
    if (e.rin == (const void*)Rin && e.d == (const void*)D && e.pairs == pairs && e.steps == steps &&
        e.sigma == sigma && e.rbytes == (int)sizeof(R))
      g = &e;
  if (!g) {
    graphs_.push_back(Graph{Rin, D, pairs, steps, (int)sizeof(R), sigma, nullptr, false});
    return run_direct<R>(Rin, D, pairs, steps, sigma, s);
  }
  if (g->direct) return run_direct<R>(Rin, D, pairs, steps, sigma, s);
  if (!g->exec) {
    if (!cap_ && cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      use_graphs_ = false;
      return run_direct<R>(Rin, D, pairs, steps, sigma, s);
    }
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    bdg_status st = BDG_OK;
    if (ok) {
      st = run_direct<R>(Rin, D, pairs, steps, sigma, cap_);
      ok = cudaStreamEndCapture(cap_, &graph) == cudaSuccess && st == BDG_OK && graph;
    }
    if (ok) ok = cudaGraphInstantiate(&g->exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      cudaGetLastError();
      if (g->exec) cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
      g->direct = true;
      return run_direct<R>(Rin, D, pairs, steps, sigma, s);
    }
  }
  BDG_CUDA_TRY(plan_, cudaGraphLaunch(g->exec, s));
  return BDG_OK;
}

template <typename RI>
template <typename R>
bdg_status InnerPCG<RI>::run_direct(const typename CT<R>::T* Rin, typename CT<R>::T* D, int pairs, int steps,
                                    double sigma, cudaStream_t s) {
  T *x = buf_[0], *r = buf_[1], *z = buf_[2], *p = buf_[3], *q = buf_[4];
  const long long n3 = 3 * np_;
  const dim3 rows(row_blocks(vlen_), pairs);
  const int dtype = sizeof(RI) == 8 ? BDG_C128 : BDG_C64;
  BDG_CUDA_TRY(plan_, (convert_pairs<R, RI>(Rin, vlen_, r, vlen_, vlen_, pairs, s)));
  bdg_status st = deflate_swapped(r, pairs, s);
  if (st) return st;
  if ((st = precondition(r, z, pairs, sigma, s)) || (st = deflate_swapped(z, pairs, s)) || (st = dots(r, z, pairs, s)))
    return st;
  k_cg_p<RI><<<rows, NT, 0, s>>>(p, z, n3, nchunk_, part_, rz_, rz_, 1);
  BDG_CUDA_TRY(plan_, cudaGetLastError());
  for (int it = 0; it < steps; ++it) {
    double* rz_cur = rz_ + (it & 1) * 4 * max_pairs_;
    double* rz_nxt = rz_ + ((it + 1) & 1) * 4 * max_pairs_;
    if ((st = apply_internal(plan_, BDG_FG, dtype, p, q, pairs, s, nullptr))) return st;
    if ((st = dots(p, q, pairs, s))) return st;
    k_cg_xr<RI><<<rows, NT, 0, s>>>(x, r, p, q, n3, nchunk_, part_, rz_cur, it == 0 ? 1 : 0);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    if (it + 1 == steps) break;
    if ((st = precondition(r, z, pairs, sigma, s)) || (st = deflate_swapped(z, pairs, s)) ||
        (st = dots(r, z, pairs, s)))
      return st;
    k_cg_p<RI><<<rows, NT, 0, s>>>(p, z, n3, nchunk_, part_, rz_cur, rz_nxt, 0);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
  }
  if (steps <= 0) {
    BDG_CUDA_TRY(plan_, (convert_pairs<RI, R>(z, vlen_, D, vlen_, vlen_, pairs, s)));
    return BDG_OK;
  }
  BDG_CUDA_TRY(plan_, (convert_pairs<RI, R>(x, vlen_, D, vlen_, vlen_, pairs, s)));
  return BDG_OK;
}

template class InnerPCG<float>;
template class InnerPCG<double>;
template bdg_status InnerPCG<float>::run_direct<float>(const float2*, float2*, int, int, double, cudaStream_t);
template bdg_status InnerPCG<float>::run_direct<double>(const double2*, double2*, int, int, double, cudaStream_t);
template bdg_status InnerPCG<double>::run_direct<double>(const double2*, double2*, int, int, double, cudaStream_t);
template bdg_status InnerPCG<float>::run<float>(const float2*, float2*, int, int, double, cudaStream_t);
template bdg_status InnerPCG<float>::run<double>(const double2*, double2*, int, int, double, cudaStream_t);
template bdg_status InnerPCG<double>::run<double>(const double2*, double2*, int, int, double, cudaStream_t);

}  // namespace bdg
