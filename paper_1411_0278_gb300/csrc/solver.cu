// Device-side GMRES for one or many independent systems and the mixed-precision
// refinement around it: per-system state, Gram-Schmidt, Givens rotations and stopping
// tests in kernels, the Arnoldi steps of a cycle replayed from a CUDA graph with a
// device-side WHILE loop, and the solve sequence (right-hand side, refinement sweeps,
// output pass).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "gstate.cuh"

namespace gbi {

// ---------------------------------------------------------------------------------
// Batched GMRES with its control on the device
// ---------------------------------------------------------------------------------
//
// S independent systems (suspensions) share one launch per pass: every vector is
// component-major over all spheres [h][Ntot], sphere n belongs to system sys[n] with
// spheres [off[s], off[s+1]).  Each system has its own Krylov state, Hessenberg
// matrix, Givens rotations, tolerance test and refinement flag; a system that has
// stopped is skipped by every kernel.  A single suspension is the case S = 1.

// Device-resident state of one system's GMRES / refinement.

// sqrt(q) and 1 / sqrt(q) for q >= 0 (0 and 0 for q <= 0) from one reciprocal square root:
// on GB300 a dependent FP64 sqrt or division costs ~650 cycles, rsqrt ~430 and an FMA 64,
// and the Arnoldi step's scalar work runs on one thread between grid-wide phases
__device__ __forceinline__ void root_and_inverse(double q, double& r, double& inv) {
  if (q > 0.0) {
    inv = rsqrt(q);
    r = q * inv;
  } else {
    inv = 0.0;
    r = 0.0;
  }
}

struct GPtr {     // per-system views into the gstate buffer
  GDev* st;
  double *H, *cs, *sn, *g, *y, *nrm;
  double* cf;                 // Gram-Schmidt coefficients c_i of the current step (one round)
  double *h1p, *h2p, *nrmp;   // per-chunk partial sums of the dot products and the norm
  int* nact;                  // systems still active after the current Arnoldi step
  unsigned int* bar;          // grid barrier of the fused single-system step: count, generation, error
  double* fp;                 // its per-block partial sums (two dot-product sets and the norm)
  unsigned int* cnt;          // per system: blocks of bk_dots_fin done in the current step
  int S, m, CH;
};



// ordered pairs of system s
__device__ __forceinline__ long long sys_pairs(const int* __restrict__ off, int s) {
  const long long n = off[s + 1] - off[s];
  return n * (n - 1);
}

// Row chunks per system of the Arnoldi reductions: a few systems get one block per
// component row (so that a single suspension still spreads over many SMs), large
// batches one block per system.

GPtr gptrs(void* base, int m, int S, int CH) {
  GPtr p;
  p.S = S;
  p.m = m;
  p.CH = CH;
  p.st = reinterpret_cast<GDev*>(base);
  double* d = reinterpret_cast<double*>(base) + (size_t)S * (sizeof(GDev) / sizeof(double) + 1);
  p.H = d; d += (size_t)S * (m + 1) * m;
  p.cs = d; d += (size_t)S * (m + 1);
  p.sn = d; d += (size_t)S * (m + 1);
  p.g = d; d += (size_t)S * (m + 1);
  p.y = d; d += (size_t)S * (m + 1);
  p.cf = d; d += (size_t)S * (m + 1);
  p.nrm = d; d += (size_t)S;
  p.h1p = d; d += (size_t)S * (m + 1) * CH;
  p.h2p = d; d += (size_t)S * (m + 1) * CH;
  p.nrmp = d; d += (size_t)S * CH;
  p.nact = reinterpret_cast<int*>(d);
  d += 1;
  p.bar = reinterpret_cast<unsigned int*>(d);
  d += 2;
  p.fp = d;
  d += 21 + (size_t)kFusedBlocks * (2 * (size_t)(m + 1) + 1);
  p.cnt = reinterpret_cast<unsigned int*>(d);
  return p;
}

__device__ __forceinline__ double block_sum_256(double v) {
  __shared__ double sh[256];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  return sh[0];
}

// part[(s (m+1) + i) CH + c] = V_i . w over the component rows of chunk c of system s,
// for i <= j_s (block (s, i, c); fixed-order block reduction).  With with_norm set, slot
// i = j_s + 1 receives w . w (the one-reduction step below).
__global__ void bk_dots(const double* __restrict__ V, size_t n, const double* __restrict__ w, int Ntot, int h,
                        const int* __restrict__ off, const GDev* __restrict__ st, int m, int CH, double* part,
                        int with_norm) {
  const int s = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
  const GDev& g = st[s];
  if (!g.active || i > g.j + with_norm) return;
  const double* v = i > g.j ? w : V + (size_t)i * n;
  const int lo = off[s], hi = off[s + 1];
  const int q0 = c * h / CH, q1 = (c + 1) * h / CH;
  double acc = 0.0;
  for (int q = q0; q < q1; ++q) {
    const size_t b = (size_t)q * Ntot;
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) acc += v[b + p] * w[b + p];
  }
  const double t = block_sum_256(acc);
  if (threadIdx.x == 0) part[((size_t)s * (m + 1) + i) * CH + c] = t;
}

// w -= sum_{i <= j_s} coef[s][i] V_i with coef[s][i] = sum over the CH chunk partials (in
// order).  A block whose spheres all belong to one system sums the partials once into
// shared memory; otherwise every thread sums them for its own system.
__global__ void bk_sub(const double* __restrict__ V, size_t n, double* w, int Ntot, const int* __restrict__ sys,
                       const GDev* __restrict__ st, int m, int CH, const double* __restrict__ part) {
  __shared__ double sc[kMaxRestart + 1];
  const int p0 = blockIdx.x * blockDim.x;
  const int pl = min(Ntot - 1, p0 + (int)blockDim.x - 1);
  const int sb = sys[p0];
  const bool uniform = sys[pl] == sb;
  if (uniform) {
    const GDev& g = st[sb];
    if (!g.active) return;
    for (int i = threadIdx.x; i <= g.j; i += blockDim.x) {
      const double* q = part + ((size_t)sb * (m + 1) + i) * CH;
      double acc = 0.0;
      for (int c = 0; c < CH; ++c) acc += q[c];
      sc[i] = acc;
    }
    __syncthreads();
  }
  const int p = p0 + threadIdx.x;
  if (p >= Ntot) return;
  const int s = sys[p];
  const GDev& g = st[s];
  if (!g.active) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  double acc = w[t];
  for (int i = 0; i <= g.j; ++i) {
    double c;
    if (uniform) {
      c = sc[i];
    } else {
      const double* q = part + ((size_t)s * (m + 1) + i) * CH;
      c = 0.0;
      for (int k = 0; k < CH; ++k) c += q[k];
    }
    acc -= c * V[(size_t)i * n + t];
  }
  w[t] = acc;
}

__device__ __forceinline__ bool norm_wanted(const GDev& g, int mode) {
  return !((mode == 0 && !g.active) || (mode == 1 && !g.enabled));
}

// part[s CH + c] = |x_s|^2 over the rows of chunk c (block (s, c)); mode 0: active
// systems, 1: enabled, 2: all
__global__ void bk_norm_part(const double* __restrict__ x, int Ntot, int h, const int* __restrict__ off,
                             const GDev* __restrict__ st, int mode, int CH, double* part) {
  const int s = blockIdx.x, c = blockIdx.y;
  if (!norm_wanted(st[s], mode)) return;
  const int lo = off[s], hi = off[s + 1];
  const int q0 = c * h / CH, q1 = (c + 1) * h / CH;
  double acc = 0.0;
  for (int q = q0; q < q1; ++q) {
    const size_t b = (size_t)q * Ntot;
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) acc += x[b + p] * x[b + p];
  }
  const double t = block_sum_256(acc);
  if (threadIdx.x == 0) part[(size_t)s * CH + c] = t;
}

// Hessenberg column j_s, Givens rotations, residual estimate and stopping test of one
// system per block (parallel loads to shared memory, one thread sweeps the rotations).
constexpr int kGmMaxM = 128;
// Hessenberg column j of system s (col[0..j] = the two Gram-Schmidt coefficient sums,
// in shared memory, overwritten), new norm hn: apply the previous rotations, form the
// new one, update g, the residual estimate and the stopping test, store the column.
// Called by one block per system; thread 0 does the serial part.
__device__ void givens_step(const GPtr& p, int s, int j, double hn, double inv_hn, double* col, double* scs,
                            double* ssn) {
  GDev* st = p.st + s;
  const int m = p.m;
  const size_t o1 = (size_t)s * (m + 1);
  const int tid = threadIdx.x;
  // every value the serial part reads, loaded by many threads at once: a chain of
  // dependent global loads on one thread would cost an L2 round trip per link
  __shared__ double s_gj, s_ibnorm, s_tol;
  __shared__ int s_iters, s_maxit;
  for (int i = tid; i < j; i += blockDim.x) {
    scs[i] = p.cs[o1 + i];
    ssn[i] = p.sn[o1 + i];
  }
  if (tid == 32) s_gj = p.g[o1 + j];   // blocks here have 128 or 256 threads
  if (tid == 33) s_ibnorm = st->inv_bnorm;
  if (tid == 34) s_tol = st->tol;
  if (tid == 35) s_iters = st->iters;
  if (tid == 36) s_maxit = st->max_iter;
  __syncthreads();
  if (tid == 0) {
    // the previous rotations, the carried entry in a register
    double carry = col[0];
    for (int i = 0; i < j; ++i) {
      const double t2 = col[i + 1];
      col[i] = scs[i] * carry + ssn[i] * t2;
      carry = -ssn[i] * carry + scs[i] * t2;
    }
    const double hjj = carry, hj1 = hn;
    double den, inv;
    root_and_inverse(hjj * hjj + hj1 * hj1, den, inv);
    const double c = den > 0 ? hjj * inv : 1.0, sg = den > 0 ? hj1 * inv : 0.0;
    col[j] = den;
    col[j + 1] = 0.0;
    const double gj = s_gj;
    const double g1 = -sg * gj;
    const int iters = s_iters + 1;
    const double res = fabs(g1) * s_ibnorm;
    const int conv = res <= s_tol;
    const int brk = hn <= 1e-300;
    const bool stop = conv || brk || iters >= s_maxit || j + 1 >= m;
    p.cs[o1 + j] = c;
    p.sn[o1 + j] = sg;
    p.g[o1 + j + 1] = g1;
    p.g[o1 + j] = c * gj;
    st->iters = iters;
    st->kdim = j + 1;
    st->res = res;
    st->converged = conv;
    st->breakdown = brk;
    if (stop) {
      st->active = 0;
    } else {
      st->inv_hn = inv_hn;
      st->j = j + 1;
      atomicAdd(p.nact, 1);
    }
  }
  __syncthreads();
  double* H = p.H + (size_t)s * (m + 1) * m;
  for (int i = tid; i <= j + 1; i += blockDim.x) H[(size_t)i * m + j] = col[i];
}

// Column j of the Hessenberg matrix from the Gram-Schmidt partial sums and the new
// norm, then the Givens step.  two_pass: coefficients of both rounds (h1p + h2p) and
// the norm of the twice-orthogonalised vector (nrmp).  Otherwise one round: h1p holds
// c_i = V_i . w for i <= j and |w|^2 in slot j + 1, and with orthonormal V_i
// |w - sum c_i V_i|^2 = |w|^2 - sum c_i^2 (clamped at zero).
// Sum of CH chunk partials by one warp: lane c loads chunks c, c + 32, ... (all loads in
// flight together) and a fixed shuffle tree adds the lanes.  L2 loads: the partials may
// come from other blocks of the same kernel.
__device__ __forceinline__ double warp_chunk_sum(const double* a, int CH) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int c = lane; c < CH; c += 32) v += __ldcg(a + c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ void finalize_column(const GPtr& p, int s, int j, int two_pass) {
  __shared__ double col[kGmMaxM + 1], scs[kGmMaxM], ssn[kGmMaxM];
  __shared__ double s_hn, s_ihn;
  const size_t o1 = (size_t)s * (p.m + 1);
  const int top = two_pass ? j : j + 1;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // one warp per slot
  for (int i = warp; i <= top; i += nw) {
    double v = warp_chunk_sum(p.h1p + (o1 + i) * p.CH, p.CH);
    if (two_pass) v += warp_chunk_sum(p.h2p + (o1 + i) * p.CH, p.CH);
    if ((threadIdx.x & 31) == 0) col[i] = v;
  }
  double nrm2 = 0.0;
  if (two_pass && warp == 0) nrm2 = warp_chunk_sum(p.nrmp + (size_t)s * p.CH, p.CH);
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm = nrm2;
    if (!two_pass) {
      nrm = col[j + 1];
      for (int i = 0; i <= j; ++i) nrm -= col[i] * col[i];
    }
    root_and_inverse(nrm, s_hn, s_ihn);
  }
  // the coefficients before the rotations act on them (one-round step: bk_sub_scale)
  for (int i = threadIdx.x; i <= j; i += blockDim.x) p.cf[o1 + i] = col[i];
  __syncthreads();
  givens_step(p, s, j, s_hn, s_ihn, col, scs, ssn);
}

__global__ void bk_finalize(GPtr p, int two_pass) {
  const int s = blockIdx.x;
  const GDev* st = p.st + s;
  if (!st->active) return;
  finalize_column(p, s, st->j, two_pass);
}

// One-reduction Arnoldi step, first half, for fewer than 64 systems: block (s, i, c)
// forms V_i . w (w . w for i = j_s + 1) over the component rows of chunk c of system s,
// as bk_dots does.  Every block of an active system, with a slot or without, counts
// itself in cnt[s] after its partial is stored; the last one sums the partials (chunk
// order) and runs the Givens step.  All blocks read j_s and the active flag before they
// count, so none can see the state the last block writes.
__global__ void __launch_bounds__(256) bk_dots_fin(const double* __restrict__ V, size_t n,
                                                   const double* __restrict__ w, int Ntot, int h,
                                                   const int* __restrict__ off, GPtr p) {
  pdl_wait();
  const int s = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
  const GDev* st = p.st + s;
  if (!st->active) return;
  const int j = st->j, CH = p.CH;
  if (i <= j + 1) {
    const double* v = i > j ? w : V + (size_t)i * n;
    const int lo = off[s], hi = off[s + 1];
    const int q0 = c * h / CH, q1 = (c + 1) * h / CH;
    double acc = 0.0;
    for (int q = q0; q < q1; ++q) {
      const size_t b = (size_t)q * Ntot;
      for (int t = lo + threadIdx.x; t < hi; t += blockDim.x) acc += v[b + t] * w[b + t];
    }
    // lanes by a shuffle tree, then the warps in order
    __shared__ double s_w[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = s_w[0];
      for (int k = 1; k < (int)(blockDim.x >> 5); ++k) tot += s_w[k];
      p.h1p[((size_t)s * (p.m + 1) + i) * CH + c] = tot;
    }
  }
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(p.cnt + s, 1u) == gridDim.y * gridDim.z - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) p.cnt[s] = 0u;
  finalize_column(p, s, j, 0);
}

// One-reduction Arnoldi step, first half, for batches of many small systems: one block
// per system, its warp k taking the slots i = k, k + 8, ... <= j_s + 1 (V_i . w, and w . w
// for i = j_s + 1) over the system's whole vector (lanes stride its elements, a shuffle
// tree adds them), then the Hessenberg column and the Givens step in the same block -- one
// block per system instead of one per (system, slot), and no counting across blocks.
__global__ void __launch_bounds__(256) bk_dots_sys(const double* __restrict__ V, size_t n,
                                                   const double* __restrict__ w, int Ntot, int h,
                                                   const int* __restrict__ off, GPtr p) {
  const int s = blockIdx.x;
  const GDev* st = p.st + s;
  if (!st->active) return;
  const int j = st->j;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int lo = off[s], ns = off[s + 1] - lo;
  const int len = ns * h;
  __shared__ double col[kGmMaxM + 1], scs[kGmMaxM], ssn[kGmMaxM];
  __shared__ double s_hn, s_ihn;
  for (int i = warp; i <= j + 1; i += nw) {
    const double* v = i > j ? w : V + (size_t)i * n;
    double acc = 0.0;
    for (int e = lane; e < len; e += 32) {
      const int q = e / ns;
      const size_t t = (size_t)q * Ntot + lo + (e - q * ns);
      acc += v[t] * w[t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) col[i] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm = col[j + 1];
    for (int i = 0; i <= j; ++i) nrm -= col[i] * col[i];
    root_and_inverse(nrm, s_hn, s_ihn);
  }
  const size_t o1 = (size_t)s * (p.m + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) p.cf[o1 + i] = col[i];
  __syncthreads();
  givens_step(p, s, j, s_hn, s_ihn, col, scs, ssn);
}

// Arnoldi source of the next pair pass, written by the kernels that produce V_j:
// FP32 records (PairArgs::x32, ncp floats per sphere, zero padding) or FP64
// component-major, both scaled by the column multipliers minv.
struct SrcOut {
  float* rec;
  double* dbl;
  int ncp;
  Scales minv;
};

__device__ __forceinline__ void write_src(const SrcOut& o, int Ntot, int h, int q, int p, double v) {
  if (o.rec != nullptr) {
    float* r = o.rec + (size_t)p * o.ncp;
    r[q] = float(v * o.minv.v[q]);
    if (q == 0)
      for (int k = h; k < o.ncp; ++k) r[k] = 0.f;
  } else if (o.dbl != nullptr) {
    o.dbl[(size_t)q * Ntot + p] = v * o.minv.v[q];
  }
}

// End of one device-looped Arnoldi step: inside the cycle graph the step's last kernel
// keeps the loop going while any system is still active (the WHILE node reads the value
// set here) and resets the count; its first thread does it before any block can leave.
// When the loop body holds several Arnoldi steps, the steps before the last only reset
// the count (on = 1); the last one (on = 2) also sets the condition and counts the trip.
struct LoopCtl {
  int* nact;
  cudaGraphConditionalHandle h;
  int on;
  long long* steps;   // optional count of loop iterations
};

__device__ __forceinline__ void loop_continue(const LoopCtl& lc) {
  if (lc.on && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    const int v = *lc.nact;
    *lc.nact = 0;
    if (lc.on == 2) {
      if (lc.steps != nullptr) *lc.steps += 1;
      cudaGraphSetConditional(lc.h, v > 0 ? 1u : 0u);
    }
  }
}

// V_{j_s} = w / h for the newly advanced j_s (and its Arnoldi source)
__global__ void bk_scale(double* V, size_t n, const double* __restrict__ w, int Ntot, const int* __restrict__ sys,
                         const GDev* __restrict__ st, SrcOut src, LoopCtl lc) {
  loop_continue(lc);
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ntot) return;
  const GDev& g = st[sys[p]];
  if (!g.active) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  const double v = w[t] * g.inv_hn;
  V[(size_t)g.j * n + t] = v;
  write_src(src, Ntot, gridDim.y, blockIdx.y, p, v);
}

// One-reduction step, after the Givens step advanced j_s: V_{j_s} = (w - sum_{i < j_s}
// c_i V_i) / h_{j_s, j_s - 1} with the coefficients cf the Givens step stored (copied
// once per block into shared memory when the block's spheres all belong to one system),
// and its source.
__global__ void bk_sub_scale(double* V, size_t n, const double* __restrict__ w, int Ntot,
                             const int* __restrict__ sys, const GDev* __restrict__ st, int m,
                             const double* __restrict__ cf, SrcOut src, LoopCtl lc) {
  pdl_wait();
  loop_continue(lc);
  __shared__ double sc[kMaxRestart + 1];
  const int p0 = blockIdx.x * blockDim.x;
  const int pl = min(Ntot - 1, p0 + (int)blockDim.x - 1);
  const int sb = sys[p0];
  const bool uniform = sys[pl] == sb;
  if (uniform) {
    const GDev& g = st[sb];
    if (!g.active) return;
    for (int i = threadIdx.x; i < g.j; i += blockDim.x) sc[i] = cf[(size_t)sb * (m + 1) + i];
    __syncthreads();
  }
  const int p = p0 + threadIdx.x;
  if (p >= Ntot) return;
  const int s = sys[p];
  const GDev& g = st[s];
  if (!g.active) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  double acc = w[t];
#pragma unroll 8
  for (int i = 0; i < g.j; ++i) {
    const double c = uniform ? sc[i] : cf[(size_t)s * (m + 1) + i];
    acc -= c * V[(size_t)i * n + t];
  }
  const double v = acc * g.inv_hn;
  V[(size_t)g.j * n + t] = v;
  write_src(src, Ntot, gridDim.y, blockIdx.y, p, v);
}

// ---------------------------------------------------------------------------------
// Fused Arnoldi step of a single system: both Gram-Schmidt rounds, the norm, the
// Givens update and V_{j+1} (with its pair-pass source) in one kernel of kFusedBlocks
// blocks, each owning a contiguous slice of the vectors, separated by three grid-wide
// barriers.  Partial sums are combined in block order by every block (identical
// results everywhere), so the result does not depend on timing.  The blocks must be
// co-resident: the kernel is launched cooperatively (64 blocks of 256 threads), so the
// launch either places every block at once or fails.  Each barrier wait is bounded as
// well; a block that gives up records an error (bar[2]) and returns, and the host
// reports GBI_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------

constexpr long long kBarrierLimit = 1ll << 22;   // polling rounds (with back-off) per barrier

__device__ bool grid_barrier(unsigned int* bar, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = atomicAdd(&bar[1], 0u);   // generation before arriving
    __threadfence();
    int ok = 1;
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      long long it = 0;
      while (atomicAdd(&bar[1], 0u) == g) {
        if (++it > kBarrierLimit) {
          atomicExch(&bar[2], 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// sum over the block in a fixed order; the leading barrier makes back-to-back calls safe
__device__ __forceinline__ double block_sum_ordered(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  return sh[0];
}

// part[i G + b] = V_i . w over [t0, t1) for i <= j (and w . w for i = top = j + 1):
// warp k of the block takes i = k, k + nwarps, ...; lanes stride the slice and a
// shuffle tree sums them (fixed order)
__device__ __forceinline__ void slice_dots(const double* __restrict__ V, size_t n, const double* __restrict__ w,
                                           int j, int top, size_t t0, size_t t1, double* part, int G, int b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i <= top; i += nw) {
    const double* v = i > j ? w : V + (size_t)i * n;
    double acc = 0.0;
    for (size_t t = t0 + lane; t < t1; t += 32) acc += v[t] * w[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[(size_t)i * G + b] = acc;
  }
}

__global__ void __launch_bounds__(256) bk_step_fused(double* V, size_t n, double* w, int Ntot, int h, GPtr p,
                                                     SrcOut so, int two_pass) {
  __shared__ double sh[256];
  __shared__ double c1[kGmMaxM + 1], c2[kGmMaxM + 1], scs[kGmMaxM], ssn[kGmMaxM];
  __shared__ double s_hn, s_ihn;
  __shared__ int s_ok;
  const GDev* st = p.st;
  if (!st->active) return;   // the same decision in every block: nothing writes the state yet
  const int j = st->j, m = p.m;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const size_t L = (n + G - 1) / G;
  const size_t t0 = (size_t)b * L, t1 = min(n, t0 + L);
  double* part1 = p.fp;
  double* part2 = p.fp + (size_t)(m + 1) * G;
  double* partn = p.fp + 2 * (size_t)(m + 1) * G;
  // (A) partial V_i . w: warp w of the block takes i = w, w + 8, ... (no block barrier)
  slice_dots(V, n, w, j, two_pass ? j : j + 1, t0, t1, part1, G, b);
  if (!grid_barrier(p.bar, &s_ok)) return;
  if (!two_pass) {
    // one round: h_{j+1,j}^2 = |w|^2 - sum c_i^2, V_{j+1} = (w - sum c_i V_i) / h_{j+1,j}
    for (int i = tid; i <= j + 1; i += blockDim.x) {
      double c = 0.0;
      for (int q = 0; q < G; ++q) c += part1[(size_t)i * G + q];
      c1[i] = c;
    }
    __syncthreads();
    if (tid == 0) {
      double nrm = c1[j + 1];
      for (int i = 0; i <= j; ++i) nrm -= c1[i] * c1[i];
      root_and_inverse(nrm, s_hn, s_ihn);
    }
    __syncthreads();
    const double hn = s_hn;
    const double inv = hn > 1e-300 ? s_ihn : 0.0;
    for (size_t t = t0 + tid; t < t1; t += blockDim.x) {
      double a = w[t];
      for (int i = 0; i <= j; ++i) a -= c1[i] * V[(size_t)i * n + t];
      const double v = a * inv;
      V[(size_t)(j + 1) * n + t] = v;
      const int q = int(t / (size_t)Ntot);
      write_src(so, Ntot, h, q, int(t - (size_t)q * Ntot), v);
    }
    if (b == 0) givens_step(p, 0, j, hn, s_ihn, c1, scs, ssn);
    return;
  }
  // (B) w1 = w - sum c1_i V_i on the slice, then partial V_i . w1
  for (int i = tid; i <= j; i += blockDim.x) {
    double c = 0.0;
    for (int q = 0; q < G; ++q) c += part1[(size_t)i * G + q];
    c1[i] = c;
  }
  __syncthreads();
  for (size_t t = t0 + tid; t < t1; t += blockDim.x) {
    double a = w[t];
    for (int i = 0; i <= j; ++i) a -= c1[i] * V[(size_t)i * n + t];
    w[t] = a;
  }
  __syncthreads();
  slice_dots(V, n, w, j, j, t0, t1, part2, G, b);
  if (!grid_barrier(p.bar, &s_ok)) return;
  // (C) w2 = w1 - sum c2_i V_i, partial |w2|^2
  for (int i = tid; i <= j; i += blockDim.x) {
    double c = 0.0;
    for (int q = 0; q < G; ++q) c += part2[(size_t)i * G + q];
    c2[i] = c;
  }
  __syncthreads();
  double nacc = 0.0;
  for (size_t t = t0 + tid; t < t1; t += blockDim.x) {
    double a = w[t];
    for (int i = 0; i <= j; ++i) a -= c2[i] * V[(size_t)i * n + t];
    w[t] = a;
    nacc += a * a;
  }
  nacc = block_sum_ordered(nacc, sh);
  if (tid == 0) partn[b] = nacc;
  if (!grid_barrier(p.bar, &s_ok)) return;
  // (D) h_{j+1,j} = |w2|, V_{j+1} = w2 / h and its source; block 0 updates the rotations
  if (tid == 0) {
    double nrm = 0.0;
    for (int q = 0; q < G; ++q) nrm += partn[q];
    root_and_inverse(nrm, s_hn, s_ihn);
  }
  __syncthreads();
  const double hn = s_hn;
  const double inv = hn > 1e-300 ? s_ihn : 0.0;
  for (size_t t = t0 + tid; t < t1; t += blockDim.x) {
    const double v = w[t] * inv;
    V[(size_t)(j + 1) * n + t] = v;
    const int q = int(t / (size_t)Ntot);
    write_src(so, Ntot, h, q, int(t - (size_t)q * Ntot), v);
  }
  if (b == 0) {
    for (int i = tid; i <= j; i += blockDim.x) c1[i] += c2[i];
    __syncthreads();
    givens_step(p, 0, j, hn, s_ihn, c1, scs, ssn);
  }
}

// start of a GMRES cycle for system s (enabled systems): beta = |V_0|, g = (beta, 0, ...);
// `first` marks the first cycle of an inner solve (the counters restart)
__device__ void init_cycle_sys(const GPtr& p, int s, int first) {
  GDev* st = p.st + s;
  const int m = p.m;
  if (first) {
    st->iters = 0;
    st->it0 = 0;
  }
  st->j = 0;
  st->kdim = 0;
  st->breakdown = 0;
  if (!st->enabled || (!first && st->converged)) {
    st->active = 0;
    return;
  }
  double beta, ibeta;
  root_and_inverse(p.nrm[s], beta, ibeta);
  if (first) {
    st->bnorm = beta;
    st->inv_bnorm = ibeta;
  }
  st->beta = beta;
  double* g = p.g + (size_t)s * (m + 1);
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  st->res = beta * st->inv_bnorm;
  st->converged = st->res <= st->tol;
  st->active = (!st->converged && st->iters < st->max_iter && beta > 0) ? 1 : 0;
  st->inv_hn = ibeta;
}


__global__ void bk_scale0(double* V0, int Ntot, const int* __restrict__ sys, const GDev* __restrict__ st,
                          SrcOut src) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ntot) return;
  const GDev& g = st[sys[p]];
  if (!g.active) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  const double v = V0[t] * g.inv_hn;
  V0[t] = v;
  write_src(src, Ntot, gridDim.y, blockIdx.y, p, v);
}

// End of a GMRES cycle in the solve graph, once every system's cycle is over: count the
// cycle's pair passes (the V_0 pass when it ran, the Arnoldi steps each system took) and
// keep the restart loop going while some system needs another cycle.  One block.
__device__ void cycle_end_all(const GPtr& p, const int* __restrict__ off, DSolve* d, cudaGraphConditionalHandle hr) {
  __shared__ unsigned long long sp;
  __shared__ int slive;
  if (threadIdx.x == 0) {
    sp = 0ull;
    slive = 0;
  }
  __syncthreads();
  const int v0_ran = d->notfirst;
  unsigned long long c = 0;
  int live = 0, any = 0;
  for (int s = threadIdx.x; s < p.S; s += blockDim.x) {
    GDev* st = p.st + s;
    const unsigned long long np = (unsigned long long)sys_pairs(off, s);
    const int iters = __ldcg(&st->iters);
    if (v0_ran && st->enabled) c += np;
    const int dd = iters - st->it0;
    st->it0 = iters;
    c += (unsigned long long)dd * np;
    live = max(live, dd);
    if (st->enabled && st->kdim > 0 && !st->converged && !st->breakdown && iters < st->max_iter) any = 1;
  }
  atomicAdd(&sp, c);
  atomicMax(&slive, live);
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    d->pairs += (long long)sp;
    d->mv32 += slive + (v0_ran ? 1 : 0);
    d->cycles += 1;
    d->first = 0;
    d->notfirst = 1;
    cudaGraphSetConditional(hr, any ? 1u : 0u);
  }
}

constexpr int kSolveSmemK = 48;   // Krylov dimensions whose triangle bk_solve_y stages in shared memory

// y_s = H_s^-1 g_s on the kdim leading rows (column-oriented back substitution).  In the
// solve graph (d set) the last system's block (counted in cnt[S]) then ends the cycle
// (cycle_end_all).
__global__ void bk_solve_y(GPtr p, DSolve* d = nullptr, const int* __restrict__ off = nullptr,
                           cudaGraphConditionalHandle hr = 0) {
  const int s = blockIdx.x;
  const GDev* st = p.st + s;
  const int k = st->kdim, m = p.m;
  const double* H = p.H + (size_t)s * (m + 1) * m;
  const size_t o1 = (size_t)s * (m + 1);
  __shared__ double rhs[kGmMaxM], yv[kGmMaxM];
  if (k > 0 && k <= kSolveSmemK) {
    // the k x k triangle in shared memory (all its loads in flight together), then the
    // substitution on the first warp
    __shared__ double Hs[kSolveSmemK * kSolveSmemK];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int r = e / k, c = e - r * k;
      if (c >= r) Hs[e] = H[(size_t)r * m + c];
    }
    __shared__ double idg[kSolveSmemK];
    for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = p.g[o1 + i];
    __syncthreads();
    // the reciprocals of the diagonal all at once, off the serial chain
    for (int i = threadIdx.x; i < k; i += blockDim.x) idg[i] = 1.0 / Hs[i * k + i];
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int i = k - 1; i >= 0; --i) {
        if (lane == 0) yv[i] = rhs[i] * idg[i];
        __syncwarp();
        const double yi = yv[i];
        for (int r = lane; r < i; r += 32) rhs[r] -= Hs[r * k + i] * yi;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) p.y[o1 + i] = yv[i];
  } else if (k > 0) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = p.g[o1 + i];
    __syncthreads();
    for (int i = k - 1; i >= 0; --i) {
      if (threadIdx.x == 0) yv[i] = rhs[i] * (1.0 / H[(size_t)i * m + i]);
      __syncthreads();
      for (int r = threadIdx.x; r < i; r += blockDim.x) rhs[r] -= H[(size_t)r * m + i] * yv[i];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) p.y[o1 + i] = yv[i];
  }
  if (d == nullptr) return;
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(p.cnt + p.S, 1u) == (unsigned int)p.S - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) p.cnt[p.S] = 0u;
  cycle_end_all(p, off, d, hr);
}

// u += minv * sum_{i < kdim_s} y_s[i] V_i  (systems whose cycle ran)
__global__ void bk_update(const double* __restrict__ V, size_t n, int Ntot, const int* __restrict__ sys, GPtr p,
                          Scales minv, double* u) {
  const int pp = blockIdx.x * blockDim.x + threadIdx.x;
  if (pp >= Ntot) return;
  const int s = sys[pp];
  const int k = p.st[s].kdim;
  if (k == 0) return;
  const size_t t = (size_t)blockIdx.y * Ntot + pp;
  const double* y = p.y + (size_t)s * (p.m + 1);
  double acc = 0.0;
  for (int i = 0; i < k; ++i) acc += y[i] * V[(size_t)i * n + t];
  u[t] += minv.v[blockIdx.y] * acc;
}

// refinement bookkeeping of system s: mode 0 stores |b_s| (from nrm), mode 1 sets rel and
// enabled, mode 2 sets rel only (the FP32 residual of a warm start's guess, which sizes
// the first inner solve but decides nothing: only the high-precision residual may stop a
// system)
__device__ void refine_sys(const GPtr& p, int s, int mode, double rtol) {
  GDev* st = p.st + s;
  double v, iv;
  root_and_inverse(p.nrm[s], v, iv);
  if (mode == 0) {
    st->nb = v;
    st->inv_nb = iv;
    st->enabled = v > 0 ? 1 : 0;
    st->rel = v > 0 ? 1.0 : 0.0;
  } else if (st->enabled) {
    st->rel = v * st->inv_nb;
    if (mode == 1) st->enabled = st->rel > rtol ? 1 : 0;
  }
}


// What follows the norms of bk_norm_then, per system (see there).
enum NormFollow : int {
  kFollowNone = 0, kFollowCycle = 1, kFollowRefine0 = 2, kFollowRefine1 = 3, kFollowSweep = 4, kFollowWarm = 5
};

struct NormCtl {
  int follow;                        // NormFollow
  int first;                         // kFollowCycle: first cycle of the solve (when d is null)
  double rtol;                       // refinement tolerance
  DSolve* d;                         // solve graph record, or null
  cudaGraphConditionalHandle ha;     // kFollowCycle in the graph: the Arnoldi loop
  cudaGraphConditionalHandle hsw;    // kFollowSweep: the sweep loop and the inner-solve IF
  cudaGraphConditionalHandle hif;
  int max_refine, max_iter;
  int incr;                          // kFollowSweep: residuals after the first sweep are updates
};

// |x_s|^2 per system (partials per row chunk as bk_norm_part forms them, added by one warp
// in a fixed order), followed in the same kernel by what uses it: every block (s, c) counts
// itself in cnt[s] once its partial is stored, and the last one of system s forms nrm[s]
// and runs the follow-up of s -- the start of a GMRES cycle (init_cycle_sys; in the solve
// graph `first` comes from the device record and the Arnoldi loop's condition is reset to 1
// so that its body runs at least once), the refinement bookkeeping (refine_sys mode 0 or 1),
// or, in the solve graph, the bookkeeping of a sweep: refine_sys mode 1, the residual pass's
// counters and, in the last system to finish (counted in cnt[S]), the decision to run the
// sweep's inner solve.  All blocks of s read the state they depend on before counting, so
// none sees the follow-up's writes.  The counters are zero between launches.
__global__ void __launch_bounds__(256) bk_norm_then(const double* __restrict__ x, int Ntot, int h,
                                                    const int* __restrict__ off, GPtr p, int mode, NormCtl nc) {
  const int s = blockIdx.x, c = blockIdx.y, CH = p.CH;
  if (nc.follow == kFollowCycle && s == 0 && c == 0 && threadIdx.x == 0) {
    *p.nact = 0;
    if (nc.d != nullptr) cudaGraphSetConditional(nc.ha, 1u);
  }
  const GDev* st = p.st + s;
  const bool want = norm_wanted(*st, mode);
  const int enabled0 = st->enabled;
  if (want) {
    const int lo = off[s], hi = off[s + 1];
    const int q0 = c * h / CH, q1 = (c + 1) * h / CH;
    double acc = 0.0;
    for (int q = q0; q < q1; ++q) {
      const size_t b = (size_t)q * Ntot;
      for (int t = lo + threadIdx.x; t < hi; t += blockDim.x) acc += x[b + t] * x[b + t];
    }
    const double t = block_sum_256(acc);
    if (threadIdx.x == 0) p.nrmp[(size_t)s * CH + c] = t;
  }
  __shared__ int s_last, s_glob;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(p.cnt + s, 1u) == (unsigned int)CH - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    const double v = want ? warp_chunk_sum(p.nrmp + (size_t)s * CH, CH) : 0.0;
    if (threadIdx.x == 0 && want) p.nrm[s] = v;
  }
  if (threadIdx.x == 0) {
    p.cnt[s] = 0u;
    switch (nc.follow) {
      case kFollowCycle: init_cycle_sys(p, s, nc.d != nullptr ? nc.d->first : nc.first); break;
      case kFollowRefine0: refine_sys(p, s, 0, nc.rtol); break;
      case kFollowRefine1:
      case kFollowSweep: refine_sys(p, s, 1, nc.rtol); break;
      case kFollowWarm: refine_sys(p, s, 2, nc.rtol); break;
      default: break;
    }
    s_glob = 0;
    if (nc.follow == kFollowSweep) {
      if (enabled0) atomicAdd(reinterpret_cast<unsigned long long*>(&nc.d->pairs), (unsigned long long)sys_pairs(off, s));
      __threadfence();
      s_glob = atomicAdd(p.cnt + p.S, 1u) == (unsigned int)p.S - 1;
    }
  }
  __syncthreads();
  if (!s_glob) return;
  // the sweep decision, once every system's refinement flag is final
  __threadfence();
  int any = 0;
  for (int q = threadIdx.x; q < p.S; q += blockDim.x) any |= __ldcg(&p.st[q].enabled);
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    p.cnt[p.S] = 0u;
    DSolve* d = nc.d;
    // the residual just tested: the high-precision pass (the first sweep, or every sweep
    // without updates) or the FP32 update r -= A_32 d of the previous sweep's inner solve
    if (nc.incr && d->refinements > 0)
      d->mv32 += 1;
    else
      d->mv64 += 1;
    d->refinements += 1;
    const int go = any && d->refinements < nc.max_refine && d->iters < nc.max_iter;
    d->ifs += go;
    cudaGraphSetConditional(nc.hif, go ? 1u : 0u);
    cudaGraphSetConditional(nc.hsw, go ? 1u : 0u);
  }
}

// x += d on enabled systems
__global__ void bk_axpy_enabled(const double* __restrict__ d, int Ntot, const int* __restrict__ sys,
                                const GDev* __restrict__ st, double* x) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ntot) return;
  if (!st[sys[p]].enabled) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  x[t] += d[t];
}

// Restarted right-preconditioned GMRES(m) on every active system of the batch for
// G^HH u = rhs (internal coordinates).  u holds the initial guess (zero or warm).
// Arnoldi (classical Gram-Schmidt twice), Givens rotations, the stopping tests and
// the triangular solves run on the device in FP64; the host launches the iterations
// in chunks (replayed from a CUDA graph when the stream allows capture) and reads the
// systems' small states once per chunk.
gbi_status gmres_batch(gbi_ctx* ctx, const Setup& s, const Batch& B, int precision, const double* rhs, double* u,
                       bool u_is_zero, double tol, int restart, int max_iter, gbi_info* info, int& iters,
                       double& relres, GDev* hst, int* before, unsigned int* bar, double outer_rtol = 0.0);

// Where the kernels producing V_j put the next pair pass's source (see SrcOut).
SrcOut src_out(const Setup& s, int precision, void* xsrc) {
  SrcOut o;
  o.rec = precision == 1 ? static_cast<float*>(xsrc) : nullptr;
  o.dbl = precision == 1 ? nullptr : static_cast<double*>(xsrc);
  o.ncp = (s.h + 3) & ~3;
  o.minv = s.minv;
  return o;
}

// Largest system of a batch (spheres), and the vector length up to which the one-round
// step gives each system a single block (bk_dots_sys)
int max_system(const Batch& B) {
  int mx = 0;
  for (int q = 0; q < B.S; ++q) mx = std::max(mx, B.h_off[q + 1] - B.h_off[q]);
  return mx;
}
constexpr long long kSysBlockElems = 4096;

// Gram-Schmidt of the Arnoldi step.  The FP64 solve (precision 0) orthogonalises twice
// (CGS2) and takes the norm of the result.  The FP32 inner solves of the refinement
// orthogonalise once and take the norm from |w|^2 - sum c_i^2, so that the dot products
// and the norm share one reduction: the inner solve only has to cut the residual by a
// few decades, its FP32 pair sums already limit the Arnoldi relation to about 1e-7, and
// the residual of every refinement sweep is recomputed from scratch in FP64 or
// double-float, so a lost digit there costs at most an extra sweep, never accuracy.
int two_pass_gs(int precision) { return precision == 0 ? 1 : 0; }

// Arnoldi steps per trip of a device-side loop: a trip costs about 4.5 us of conditional
// node overhead on GB300 besides its kernels, a step after its system has stopped about
// 4 us (its kernels return at once), so several steps a trip pay off.
constexpr int kArnoldiUnroll = 4;

// kChunk Arnoldi iterations of every active system: pair pass on the source of V_j
// (written by the previous bk_scale / bk_scale0 / bk_sub_scale), classical Gram-Schmidt
// (see two_pass_gs), Givens update and V_{j+1} with its source -- eight kernels per
// iteration with two rounds, four with one.  With
// fused set and a single system the seven kernels after the pair pass are replaced by
// bk_step_fused; that is faster for direct launches, while inside the cycle graph the
// separate kernels (graph launch overhead about a microsecond each) measured faster than
// the fused kernel's three grid barriers.
gbi_status launch_chunk(gbi_ctx* ctx, const Setup& s, const Batch& B, int precision, const GPtr& gp, int m,
                        double* Vb, double* w, void* xsrc, int kChunk, bool fused, LoopCtl lc = LoopCtl{}) {
  const int S = B.S, Ntot = B.Ntot, h = s.h;
  const size_t n = (size_t)Ntot * h;
  const dim3 g2((Ntot + 255) / 256, h);
  PairArgs pa = pair_args(s, precision == 1 ? nullptr : static_cast<const double*>(xsrc), w, 1.0, 0.0, 1, s.ones,
                          6);
  if (precision == 1) pa.x32 = static_cast<const float*>(xsrc);
  pa.sys_of = B.sys;
  pa.nsys = B.S;
  pa.npairs = batch_pairs(B);
  pa.sys_off = B.off;
  pa.sys_flag = &gp.st[0].active;
  pa.sys_flag_stride = int(sizeof(GDev) / sizeof(int));
  const SrcOut so = src_out(s, precision, xsrc);
  const dim3 gd(S, m + 1, gp.CH);
  const int two = two_pass_gs(precision);
  // programmatic dependent launch inside the one-reduction step, between kernels of the
  // same sequence (the first pair pass of a chunk follows other work)
  const bool pdl = ctx->pdl && !two;
  for (int c = 0; c < kChunk; ++c) {
    LoopCtl lcs = lc;
    if (lc.on) lcs.on = c + 1 < kChunk ? 1 : 2;
    pa.pdl = pdl && c > 0;
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, precision, pa));
    if (fused && S == 1) {
      // a single system launched step by step: the whole orthogonalisation in one kernel.
      // Its grid barriers need every block resident at once: a cooperative launch
      // guarantees that (or fails with cudaErrorCooperativeLaunchTooLarge) instead of
      // assuming it.
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kFusedBlocks);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = ctx->stream;
      cudaLaunchAttribute coop[1];
      coop[0].id = cudaLaunchAttributeCooperative;
      coop[0].val.cooperative = 1;
      cfg.attrs = coop;
      cfg.numAttrs = 1;
      GBI_CHECK(cudaLaunchKernelEx(&cfg, bk_step_fused, Vb, n, w, Ntot, h, gp, so, two));
      ++ctx->launches;
      continue;
    }
    if (two) {
      bk_dots<<<gd, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, h, B.off, gp.st, m, gp.CH, gp.h1p, 0);
      bk_sub<<<g2, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, B.sys, gp.st, m, gp.CH, gp.h1p);
      bk_dots<<<gd, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, h, B.off, gp.st, m, gp.CH, gp.h2p, 0);
      bk_sub<<<g2, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, B.sys, gp.st, m, gp.CH, gp.h2p);
      bk_norm_part<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(w, Ntot, h, B.off, gp.st, 0, gp.CH, gp.nrmp);
      bk_finalize<<<S, 128, 0, ctx->stream>>>(gp, 1);
      bk_scale<<<g2, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, B.sys, gp.st, so, lcs);
      ctx->launches += 7;
    } else {
      if (S < 64) {
        // dot products, norm and Givens step in one kernel
        GBI_CHECK(launch_pdl(pdl, gd, dim3(256), ctx->stream, bk_dots_fin, Vb, n, w, Ntot, h, B.off, gp));
        ++ctx->launches;
      } else if ((long long)max_system(B) * h <= kSysBlockElems) {
        // many small systems: one block each
        bk_dots_sys<<<S, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, h, B.off, gp);
        ++ctx->launches;
      } else {
        bk_dots<<<gd, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, h, B.off, gp.st, m, gp.CH, gp.h1p, 1);
        bk_finalize<<<S, 128, 0, ctx->stream>>>(gp, 0);
        ctx->launches += 2;
      }
      GBI_CHECK(launch_pdl(pdl && S < 64, g2, dim3(256), ctx->stream, bk_sub_scale, Vb, n, w, Ntot, B.sys, gp.st,
                           m, gp.cf, so, lcs));
      ++ctx->launches;
    }
  }
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

// Per-system GMRES set-up.  With outer_rtol > 0 (an inner solve of the refinement) the
// tolerance relative to the current residual r is loosened to 0.1 outer_rtol |b| / |r|
// when that is larger than tol: the solve only has to bring |r| a decade below the
// target, so a refinement sweep that starts close to it needs few iterations.
// In the solve graph (d set) the iteration cap is what the whole solve has left, the
// record marks the first cycle and the restart loop's condition starts at 1.
__global__ void bk_setup(GPtr p, double tol, int max_iter, double outer_rtol, DSolve* d = nullptr,
                         cudaGraphConditionalHandle hr = 0) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.S) return;
  GDev* st = p.st + s;
  if (d != nullptr) max_iter = (int)max(0ll, (long long)max_iter - d->iters);
  if (s == 0) {
    p.bar[0] = 0u;   // arrivals
    p.bar[2] = 0u;   // error flag
    if (d != nullptr) {
      d->first = 1;
      d->notfirst = 0;
      cudaGraphSetConditional(hr, 1u);
    }
  }
  p.cnt[s] = 0u;
  st->tol = outer_rtol > 0 ? fmax(tol, 0.1 * outer_rtol / fmax(st->rel, 1e-300)) : tol;
  st->max_iter = max_iter;
  st->m = p.m;
  st->active = 0;
  st->converged = 0;
  st->iters = 0;
}

gbi_status gmres_batch(gbi_ctx* ctx, const Setup& s, const Batch& B, int precision, const double* rhs, double* u,
                       bool u_is_zero, double tol, int restart, int max_iter, gbi_info* info, int& iters,
                       double& relres, GDev* hst, int* before, unsigned int* bar, double outer_rtol) {
  constexpr int kChunk = 6;
  const int S = B.S, Ntot = B.Ntot, h = s.h;
  const size_t n = (size_t)Ntot * h;
  const int m = std::max(1, std::min(restart, kMaxRestart));
  GBI_TRY(ensure(ctx, ctx->krylov, sizeof(double) * n * (m + 1)));
  GBI_TRY(ensure(ctx, ctx->w, sizeof(double) * n));
  GBI_TRY(ensure(ctx, ctx->gstate, sizeof(double) * gstate_doubles(m, S, arnoldi_chunks(S, h), kFusedBlocks)));
  // gathered Arnoldi source: FP64 component-major, or FP32 records of round4(h) floats
  GBI_TRY(ensure(ctx, ctx->x32, std::max(sizeof(double) * n, sizeof(float) * (size_t)Ntot * ((h + 3) & ~3))));
  double* Vb = P<double>(ctx->krylov);
  double* w = P<double>(ctx->w);
  void* xsrc = ctx->x32.p;
  const GPtr gp = gptrs(ctx->gstate.p, m, S, arnoldi_chunks(S, h));
  const dim3 g2((Ntot + 255) / 256, h);
  const int sblk = (S + 127) / 128;
  iters = 0;
  relres = 0.0;
  bk_setup<<<sblk, 128, 0, ctx->stream>>>(gp, tol, std::max(0, max_iter), outer_rtol);
  ++ctx->launches;
  // cycle graph: a WHILE node whose body is one Arnoldi step of every active system, the
  // step's last kernel setting the loop condition; the loop runs on the device until no
  // system is active, so a GMRES cycle costs one graph launch and one read of the
  // per-system states.  Built once per buffer set and replayed afterwards.
  const bool graphs = ctx->allow_graphs && ctx->stream != nullptr && !ctx->prof;
  if (graphs) {
    const void* key[8] = {Vb, w, xsrc, ctx->gstate.p, B.sys, B.off, s.pos.hi, s.pos.p64};
    const long long ikey[6] = {(long long)n, S, m, precision, s.trunc, Ntot};
    bool same = ctx->chunk_exec != nullptr;
    for (int i = 0; i < 8 && same; ++i) same = ctx->chunk_key[i] == key[i];
    for (int i = 0; i < 6 && same; ++i) same = ctx->chunk_ikey[i] == ikey[i];
    if (!same) {
      if (ctx->chunk_exec) cudaGraphExecDestroy(ctx->chunk_exec);
      ctx->chunk_exec = nullptr;
      cudaGraph_t graph = nullptr;
      GBI_CHECK(cudaGraphCreate(&graph, 0));
      cudaGraphConditionalHandle handle;
      cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node = nullptr;
      if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
      const long long saved = ctx->launches;
      gbi_status st = GBI_OK;
      if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(ctx->stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          st = launch_chunk(ctx, s, B, precision, gp, m, Vb, w, xsrc, kArnoldiUnroll, false,
                            LoopCtl{gp.nact, handle, 1, nullptr});
          cudaGraph_t body = nullptr;
          const cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &body);
          if (e == cudaSuccess) e = e2;
        }
      }
      ctx->chunk_nodes = int(ctx->launches - saved);   // kernels per loop iteration
      ctx->launches = saved;
      if (st == GBI_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ctx->chunk_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (st != GBI_OK) return st;
      GBI_CHECK(e);
      for (int i = 0; i < 8; ++i) ctx->chunk_key[i] = key[i];
      for (int i = 0; i < 6; ++i) ctx->chunk_ikey[i] = ikey[i];
    }
  }
  bool first = true;
  for (int q = 0; q < S; ++q) before[q] = 0;
  while (true) {
    // V_0 = rhs - A u on the enabled systems, beta_s = |V_0,s|
    GBI_CHECK(cudaMemcpyAsync(Vb, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (!(first && u_is_zero)) {
      PairArgs pr = pair_args(s, u, Vb, -1.0, 1.0, 1, s.ones, 6);
      pr.sys_of = B.sys;
      pr.nsys = B.S;
      pr.npairs = batch_pairs(B);
      pr.sys_off = B.off;
      pr.sys_flag = &gp.st[0].enabled;
      pr.sys_flag_stride = int(sizeof(GDev) / sizeof(int));
      GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, precision, pr));
      if (info) {
        (precision == 1 ? info->matvecs_f32 : info->matvecs_f64) += 1;
        for (int q = 0; q < S; ++q)
          if (hst[q].enabled) info->pair_interactions += (long long)(B.h_off[q + 1] - B.h_off[q]) * (B.h_off[q + 1] - B.h_off[q] - 1);
      }
    }
    {
      NormCtl nc{};
      nc.follow = kFollowCycle;
      nc.first = first ? 1 : 0;
      bk_norm_then<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(Vb, Ntot, h, B.off, gp, 1, nc);
    }
    bk_scale0<<<g2, 256, 0, ctx->stream>>>(Vb, Ntot, B.sys, gp.st, src_out(s, precision, xsrc));
    ctx->launches += 2;
    GBI_CHECK(cudaGetLastError());
    if (first)
      for (int q = 0; q < S; ++q) before[q] = 0;      // the first cycle restarts the counters
    else
      for (int q = 0; q < S; ++q) before[q] = hst[q].iters;
    first = false;
    auto account = [&](int nsteps) {
      // states after the launched steps: pair work of the systems that took them
      int live = 0;
      for (int q = 0; q < S; ++q) {
        const int d = hst[q].iters - before[q];
        before[q] = hst[q].iters;
        live = std::max(live, d);
        if (info) info->pair_interactions += (long long)d * (B.h_off[q + 1] - B.h_off[q]) * (B.h_off[q + 1] - B.h_off[q] - 1);
      }
      if (info) (precision == 1 ? info->matvecs_f32 : info->matvecs_f64) += live;
      ctx->stat_dead[precision * 9 + SET_H * 3 + SET_H] += std::max(0, nsteps - live);
      return live;
    };
    auto read_states = [&]() -> gbi_status {
      GBI_CHECK(cudaMemcpyAsync(hst, gp.st, sizeof(GDev) * S, cudaMemcpyDeviceToHost, ctx->stream));
      GBI_CHECK(cudaMemcpyAsync(bar, gp.bar, sizeof(unsigned int) * 3, cudaMemcpyDeviceToHost, ctx->stream));
      GBI_CHECK(cudaStreamSynchronize(ctx->stream));
      if (bar[2] != 0u) {
        ctx->err = "fused Arnoldi step: a grid barrier wait gave up";
        return GBI_ERR_TIMEOUT;
      }
      return GBI_OK;
    };
    if (graphs) {
      // the whole cycle's Arnoldi steps in one launch; the loop ran max(1, most steps) times
      GBI_CHECK(cudaGraphLaunch(ctx->chunk_exec, ctx->stream));
      GBI_TRY(read_states());
      int most = 0;
      for (int q = 0; q < S; ++q) most = std::max(most, hst[q].iters - before[q]);
      const int trips = std::max(1, (most + kArnoldiUnroll - 1) / kArnoldiUnroll);
      ctx->launches += (long long)trips * ctx->chunk_nodes;
      account(trips * kArnoldiUnroll);
    } else {
      // host-driven: chunks of kChunk steps with a state read after each
      GBI_TRY(read_states());
      bool any = false;
      for (int q = 0; q < S; ++q) any = any || hst[q].active;
      while (any) {
        GBI_TRY(launch_chunk(ctx, s, B, precision, gp, m, Vb, w, xsrc, kChunk, true));
        GBI_TRY(read_states());
        account(kChunk);
        any = false;
        for (int q = 0; q < S; ++q) any = any || hst[q].active;
      }
    }
    bk_solve_y<<<S, 128, 0, ctx->stream>>>(gp);
    bk_update<<<g2, 256, 0, ctx->stream>>>(Vb, n, Ntot, B.sys, gp, s.minv, u);
    ctx->launches += 2;
    GBI_CHECK(cudaGetLastError());
    bool restart_any = false;
    for (int q = 0; q < S; ++q) {
      const GDev& g = hst[q];
      iters = std::max(iters, g.iters);
      if (g.enabled && g.kdim > 0 && !g.converged && !g.breakdown && g.iters < g.max_iter) restart_any = true;
    }
    if (!restart_any) break;
  }
  relres = 0.0;
  for (int q = 0; q < S; ++q)
    if (hst[q].enabled) relres = std::max(relres, hst[q].res);
  return GBI_OK;
}

// ---------------------------------------------------------------------------------
// The whole mixed-precision solve as one CUDA graph
// ---------------------------------------------------------------------------------
//
// Every decision that solve_core's host-driven sequence takes between kernels is taken on
// the device instead: the refinement sweeps, the GMRES cycles of an inner solve and the
// Arnoldi steps of a cycle are nested WHILE nodes (an IF node skips the inner solve of a
// sweep that has met the tolerance), and the counters of gbi_info live in a DSolve record
// read back once.  The kernels and their order are those of the host-driven sequence, so
// the results are the same bit for bit.


__global__ void gk_copy(double* __restrict__ dst, const double* __restrict__ src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void gk_zero(double* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = 0.0;
}

// input guard: a centre distance below min_sep a (min_sep > 0) or a NaN / infinite input
// stops every system (the host reports GBI_ERR_OVERLAP or GBI_ERR_ARG after the graph)
__global__ void gk_guard(GPtr p, const unsigned int* __restrict__ minr2, const int* __restrict__ bad, double a,
                         double min_sep, DSolve* d) {
  const float mr2 = __uint_as_float(*minr2);
  const bool ov = min_sep > 0 && sqrt(double(mr2)) / a < min_sep;
  const bool bi = *bad != 0;
  if (!ov && !bi) return;
  for (int s = threadIdx.x; s < p.S; s += blockDim.x) p.st[s].enabled = 0;
  if (threadIdx.x == 0) {
    if (ov) d->overlap = 1;
    if (bi) d->bad_input = 1;
  }
}

// the sweep loop runs while some system still needs a correction
__global__ void gk_sweep_start(GPtr p, cudaGraphConditionalHandle hsw) {
  int any = 0;
  for (int s = threadIdx.x; s < p.S; s += blockDim.x) any |= p.st[s].enabled;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) cudaGraphSetConditional(hsw, any ? 1u : 0u);
}

// end of an inner solve: its iterations are the most any system took
__global__ void gk_gmres_end(GPtr p, DSolve* d) {
  __shared__ int smax;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  int mx = 0;
  for (int s = threadIdx.x; s < p.S; s += blockDim.x) mx = max(mx, p.st[s].iters);
  atomicMax(&smax, mx);
  __syncthreads();
  if (threadIdx.x == 0) d->iters += smax;
}

__global__ void gk_summary(GPtr p, DSolve* d) {
  __shared__ double sm[256];
  double mx = 0.0;
  for (int s = threadIdx.x; s < p.S; s += blockDim.x) mx = fmax(mx, p.st[s].rel);
  sm[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) d->rel_max = sm[0];
}

// Building the graph by stream capture: a conditional node is added to the graph that
// the current stream is capturing, and its body is captured on a stream of its own
// (one per nesting level) while the library's launches are pointed at that stream.
struct GraphBuild {
  gbi_ctx* ctx;
  cudaError_t err = cudaSuccess;
  int nopen = 0;                   // bodies being captured
  long long nested[kCapLevels + 1] = {};   // launches inside nested bodies, per depth (0: top)
  long long own[4] = {};           // launches per execution of a body kind (see BodyKind)

  bool ok(cudaError_t e) {
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    return err == cudaSuccess;
  }
  cudaGraph_t capturing() {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    if (!ok(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr))) return nullptr;
    if (cs != cudaStreamCaptureStatusActive) {
      ok(cudaErrorStreamCaptureInvalidated);
      return nullptr;
    }
    return g;
  }
  cudaGraphConditionalHandle handle() {
    cudaGraphConditionalHandle h = 0;
    cudaGraph_t g = capturing();
    if (g != nullptr) ok(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    return h;
  }
  // a conditional node after everything captured so far on the current stream
  cudaGraph_t node(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (!ok(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, &deps, nullptr, &nd))) return nullptr;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaGraphNode_t nodeh = nullptr;
    if (!ok(cudaGraphAddNode(&nodeh, g, deps, nullptr, nd, &cp))) return nullptr;
    if (!ok(cudaStreamUpdateCaptureDependencies(ctx->stream, &nodeh, nullptr, 1, cudaStreamSetCaptureDependencies)))
      return nullptr;
    return cp.conditional.phGraph_out[0];
  }
  // capture emit() into body on the next level's stream; kind: which own[] it fills
  template <typename F>
  gbi_status body(cudaGraph_t g, int kind, F&& emit) {
    const int k = nopen + 1;   // nesting depth of the new body
    if (g == nullptr || err != cudaSuccess || k > kCapLevels) return GBI_ERR_CUDA;
    cudaStream_t cs = ctx->cap[k - 1];
    if (!ok(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
      return GBI_ERR_CUDA;
    cudaStream_t outer = ctx->stream;
    nested[k] = 0;
    nopen = k;
    ctx->stream = cs;
    const long long before = ctx->launches;
    const gbi_status st = emit();
    ctx->stream = outer;
    nopen = k - 1;
    cudaGraph_t out = nullptr;
    ok(cudaStreamEndCapture(cs, &out));
    const long long total = ctx->launches - before;
    own[kind] = total - nested[k];
    nested[k - 1] += total;
    if (st != GBI_OK) return st;
    return err == cudaSuccess ? GBI_OK : GBI_ERR_CUDA;
  }
};

enum BodyKind { kBodySweep = 0, kBodyIf = 1, kBodyCycle = 2, kBodyStep = 3 };

gbi_status gmres_reserve(gbi_ctx* ctx, const Setup& s, const Batch& B, int m) {
  const size_t n = (size_t)B.Ntot * s.h;
  GBI_TRY(ensure(ctx, ctx->krylov, sizeof(double) * n * (m + 1)));
  GBI_TRY(ensure(ctx, ctx->w, sizeof(double) * n));
  GBI_TRY(ensure(ctx, ctx->gstate, sizeof(double) * gstate_doubles(m, B.S, arnoldi_chunks(B.S, s.h), kFusedBlocks)));
  GBI_TRY(ensure(ctx, ctx->x32, std::max(sizeof(double) * n, sizeof(float) * (size_t)B.Ntot * ((s.h + 3) & ~3))));
  return GBI_OK;
}

// Inner FP32 GMRES of one sweep in the solve graph: set-up, then a WHILE node over the
// cycles whose body is one cycle of gmres_batch (V_0 = rhs - A u, norms, cycle start,
// the Arnoldi WHILE node, triangular solve, update, restart decision).
gbi_status emit_gmres(GraphBuild& gb, const Setup& s, const Batch& B, const GPtr& gp, int m, const double* rhs,
                      double* u, double tol, int max_iter, double outer_rtol, DSolve* d) {
  gbi_ctx* ctx = gb.ctx;
  const int S = B.S, Ntot = B.Ntot, h = s.h;
  const size_t n = (size_t)Ntot * h;
  double* Vb = P<double>(ctx->krylov);
  double* w = P<double>(ctx->w);
  void* xsrc = ctx->x32.p;
  const dim3 g2((Ntot + 255) / 256, h);
  const int sblk = (S + 127) / 128;
  const cudaGraphConditionalHandle hr = gb.handle();
  bk_setup<<<sblk, 128, 0, ctx->stream>>>(gp, tol, max_iter, outer_rtol, d, hr);
  ++ctx->launches;
  GBI_TRY(gb.body(gb.node(hr, cudaGraphCondTypeWhile), kBodyCycle, [&]() -> gbi_status {
    gk_copy<<<grid1(n), 256, 0, ctx->stream>>>(Vb, rhs, n);
    ++ctx->launches;
    PairArgs pr = pair_args(s, u, Vb, -1.0, 1.0, 1, s.ones, 6);
    pr.sys_of = B.sys;
    pr.nsys = B.S;
    pr.npairs = batch_pairs(B);
    pr.sys_off = B.off;
    pr.sys_flag = &gp.st[0].enabled;
    pr.sys_flag_stride = int(sizeof(GDev) / sizeof(int));
    pr.active = &d->notfirst;   // u is zero in the first cycle
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, 1, pr));
    const cudaGraphConditionalHandle ha = gb.handle();
    {
      NormCtl nc{};
      nc.follow = kFollowCycle;
      nc.d = d;
      nc.ha = ha;
      bk_norm_then<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(Vb, Ntot, h, B.off, gp, 1, nc);
    }
    bk_scale0<<<g2, 256, 0, ctx->stream>>>(Vb, Ntot, B.sys, gp.st, src_out(s, 1, xsrc));
    ctx->launches += 2;
    GBI_TRY(gb.body(gb.node(ha, cudaGraphCondTypeWhile), kBodyStep, [&]() -> gbi_status {
      return launch_chunk(ctx, s, B, 1, gp, m, Vb, w, xsrc, kArnoldiUnroll, false, LoopCtl{gp.nact, ha, 1, &d->steps});
    }));
    bk_solve_y<<<S, 128, 0, ctx->stream>>>(gp, d, B.off, hr);
    bk_update<<<g2, 256, 0, ctx->stream>>>(Vb, n, Ntot, B.sys, gp, s.minv, u);
    ctx->launches += 2;
    GBI_CHECK(cudaGetLastError());
    return GBI_OK;
  }));
  gk_gmres_end<<<1, 256, 0, ctx->stream>>>(gp, d);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

// The full solve for a batch of independent suspensions (S = 1: one suspension).
// Inputs and outputs are concatenated over the systems ([Ntot][3], [Ntot][h]).
gbi_status solve_core(gbi_ctx* ctx, const gbi_params* prm, const Batch& B, const double* R, const double* Va,
                      const double* Oa, const double* VH, const double* Fe, const double* Te, double* V,
                      double* Omega, double* QH, int warm_start, gbi_info* inf, const StepHooks* hooks) {
  const int N = B.Ntot, S = B.S;
  Setup s;
  GBI_TRY(setup_call(ctx, s, N, prm->trunc, prm->a, prm->eta, R, false));
  long long pairs_all = 0;
  for (int q = 0; q < S; ++q) {
    const long long ns = B.h_off[q + 1] - B.h_off[q];
    pairs_all += ns * (ns - 1);
  }
  s.pairs_per_pass = pairs_all;
  const int D = s.D, h = s.h;
  const size_t nh = (size_t)N * h;
  const dim3 g2((N + 255) / 256, h);
  // arithmetic of the refinement residual (FP64, or double-float for precision 2 and 3)
  // and of the right-hand-side and output passes (the same, or FP32 for precision 3)
  const int hp = prm->precision >= 2 ? 2 : 0;
  const int io = prm->precision == 3 ? 1 : hp;
  // residual updates after the first refinement sweep (the double-float modes; precision 1
  // computes every sweep's residual in FP64)
  const bool incr = hp == 2;
  const int restart = std::max(1, std::min(prm->restart > 0 ? prm->restart : 40, kMaxRestart));
  GBI_TRY(ensure(ctx, ctx->xQ, sizeof(double) * (size_t)N * D));
  GBI_TRY(ensure(ctx, ctx->b, sizeof(double) * nh));
  GBI_TRY(ensure(ctx, ctx->r, sizeof(double) * nh));
  GBI_TRY(ensure(ctx, ctx->delta, sizeof(double) * nh));
  GBI_TRY(ensure(ctx, ctx->xVL, sizeof(double) * 6 * N));
  GBI_TRY(status_words(ctx));
  GBI_TRY(ensure(ctx, ctx->gstate, sizeof(double) * gstate_doubles(restart, S, arnoldi_chunks(S, h), kFusedBlocks)));
  double* xF = P<double>(ctx->xQ);              // rows 0..5 of the full vector
  double* xQH = P<double>(ctx->xQ) + (size_t)6 * N;
  double* b = P<double>(ctx->b);
  double* r = P<double>(ctx->r);
  double* dl = P<double>(ctx->delta);
  const GPtr gp = gptrs(ctx->gstate.p, restart, S, arnoldi_chunks(S, h));
  const double c2a = s.scale.v[3];
  Scales hscale;
  for (int i = 0; i < kMaxD; ++i) hscale.v[i] = (i < h) ? s.scale.v[6 + i] : 1.0;
  auto batched = [&](PairArgs p, const int* flag) {
    p.sys_of = B.sys;
    p.nsys = B.S;
    p.npairs = batch_pairs(B);
    p.sys_off = B.off;
    p.sys_flag = flag;
    p.sys_flag_stride = int(sizeof(GDev) / sizeof(int));
    return p;
  };
  // host copies of the per-system states, the barrier words, per-system counters and
  // the solve graph's record with the smallest-distance word
  const size_t hs_states = (sizeof(GDev) * (size_t)S + 15) & ~size_t(15);
  const size_t hs_rec = hs_states + 16 + ((sizeof(int) * (size_t)S + 15) & ~size_t(15));
  GBI_TRY(host_scratch(ctx, hs_rec + sizeof(DSolve) + 16));
  GDev* hst = reinterpret_cast<GDev*>(ctx->hs);
  unsigned int* hbar = reinterpret_cast<unsigned int*>(ctx->hs + hs_states);
  int* hbefore = reinterpret_cast<int*>(ctx->hs + hs_states + 16);
  DSolve* hrec = reinterpret_cast<DSolve*>(ctx->hs + hs_rec);
  unsigned int* hbits = reinterpret_cast<unsigned int*>(ctx->hs + hs_rec + sizeof(DSolve));

  // the caller's inputs -> internal coordinates: F^L and b = -8 pi eta V^H
  int* bad_in = input_error_word(ctx);
  // centres and packed inputs; a NaN or infinite value in R, V^H, F^e or T^e (or V^a,
  // Omega^a, read at the end) sets the input word, cleared here first
  auto pack_inputs = [&]() -> gbi_status {
    GBI_CHECK(cudaMemsetAsync(bad_in, 0, sizeof(int), ctx->stream));
    GBI_TRY(launch_positions(ctx, s, R, bad_in));
    k_pack_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, c2a, Fe, Te, xF, bad_in);
    k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, VH, hscale, -8.0 * kPi * s.eta, b, bad_in);
    ctx->launches += 2;
    GBI_CHECK(cudaGetLastError());
    return GBI_OK;
  };
  // b -= G^HL F^L, with the overlap scan
  auto rhs_pass = [&]() -> gbi_status {
    GBI_CHECK(cudaMemsetAsync(ctx->minr2.p, 0x7f, sizeof(unsigned int), ctx->stream));   // a huge float
    PairArgs p = batched(pair_args(s, xF, b, -1.0, 1.0, 0, s.ones, 0), nullptr);
    p.min_r2_bits = P<unsigned int>(ctx->minr2);
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_L, io, p));
    return GBI_OK;
  };
  // 8 pi eta x^{V,L} = -(G^LL F^L + G^LH Q^H) incl. self
  auto output_pass = [&]() -> gbi_status {
    PairArgs p = batched(pair_args(s, P<double>(ctx->xQ), P<double>(ctx->xVL), -1.0 / (8.0 * kPi * s.eta), 0.0, 1,
                                   s.ones, 0),
                         nullptr);
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_L, SET_ALL, io, p));
    return GBI_OK;
  };
  // internal coordinates -> the caller's V, Omega (and Q^H)
  auto unpack_outputs = [&]() -> gbi_status {
    k_finalize_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, c2a, P<double>(ctx->xVL), Va, Oa, V, Omega, bad_in);
    ++ctx->launches;
    if (QH) {
      k_unpack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, xQH, hscale, QH);
      ++ctx->launches;
    }
    GBI_CHECK(cudaGetLastError());
    return GBI_OK;
  };
  const int max_iter = prm->max_iter > 0 ? prm->max_iter : 1000;
  const double rtol = prm->rtol > 0 ? prm->rtol : 1e-10;
  const double inner = prm->inner_rtol > 0 ? prm->inner_rtol : 1e-5;
  const int max_refine = prm->max_refine > 0 ? prm->max_refine : 8;

  // ---- the mixed-precision solve as one graph (see GraphBuild): every device step of
  // the sequence below, the decisions taken by kernels instead of the host
  // (a warm start replays the graph too, with the guess packed ahead of it; a trap step
  // with its hooks and a warm start takes the host-driven sequence)
  const bool warm = warm_start != 0;
  if (prm->precision >= 1 && (!warm || hooks == nullptr) && ctx->allow_graphs && ctx->stream != nullptr &&
      !ctx->prof) {
    auto bits = [](double v) {
      long long b;
      std::memcpy(&b, &v, sizeof(b));
      return b;
    };
    // the graph reads and writes only the context's own buffers (the caller's arrays are
    // packed before it and unpacked after it), so the key holds none of the caller's
    // every buffer the graph touches at its final size first (a repeated call then
    // allocates nothing): the Krylov workspace, the device record, and the source
    // records of every FP32 / double-float pass (right-hand side, residual, outputs)
    GBI_TRY(gmres_reserve(ctx, s, B, restart));
    GBI_TRY(ensure(ctx, ctx->dsolve, sizeof(DSolve)));
    {
      size_t x32b = ctx->x32.bytes;
      const int pass_cols[3] = {SET_L, SET_H, SET_ALL};
      const int pass_prec[3] = {io, hp, io};
      for (int i = 0; i < 3; ++i)
        if (pass_prec[i] >= 1)
          x32b = std::max(x32b, sizeof(float) * (size_t)rec_floats(ncols_of(s.trunc, pass_cols[i]), pass_prec[i] == 2) *
                                    (size_t)N);
      GBI_TRY(ensure(ctx, ctx->x32, x32b));
    }
    const void* ptrs[] = {B.sys, B.off, ctx->pos_hi.p, ctx->pos_lo.p, ctx->pos64.p, ctx->xQ.p, ctx->b.p, ctx->r.p, ctx->delta.p, ctx->xVL.p, ctx->minr2.p,
                          ctx->krylov.p, ctx->w.p, ctx->x32.p, ctx->gstate.p, ctx->dsolve.p, ctx->tile.p, ctx->tilecnt.p};
    std::vector<long long> key = {N, S, pairs_all, max_system(B), prm->trunc, prm->precision, restart, max_iter,
                                  max_refine,
                                  bits(rtol), bits(inner), bits(prm->min_sep), bits(prm->a), bits(prm->eta),
                                  ctx->wpt_gen, ctx->force_wpt, warm ? 1 : 0};
    for (const void* q : ptrs) key.push_back((long long)(uintptr_t)q);
    if (hooks != nullptr) {
      // the caller's work and arrays go into the graph as well
      const void* io[] = {R, Va, Oa, VH, Fe, Te, V, Omega, QH};
      key.push_back(-1);
      for (const void* q : io) key.push_back((long long)(uintptr_t)q);
      key.insert(key.end(), hooks->key.begin(), hooks->key.end());
    }
    const bool ready = ctx->solve_exec != nullptr && key == ctx->solve_key;
    const bool build = !ready && key == ctx->solve_prev && key != ctx->solve_failed;
    ctx->solve_prev = key;
    if (build) {
      // a repeated call: its buffers already have their sizes, so nothing below allocates
      bool built = false;
      {
        bool streams = true;
        for (int i = 0; i < kCapLevels && streams; ++i)
          if (!ctx->cap[i]) streams = cudaStreamCreateWithFlags(&ctx->cap[i], cudaStreamNonBlocking) == cudaSuccess;
        if (streams) {
          if (ctx->solve_exec) cudaGraphExecDestroy(ctx->solve_exec);
          ctx->solve_exec = nullptr;
          DSolve* d = P<DSolve>(ctx->dsolve);
          GraphBuild gb{ctx};
          const long long saved = ctx->launches;
          gbi_status st = GBI_ERR_CUDA;
          cudaGraph_t graph = nullptr;
          if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            st = [&]() -> gbi_status {
              GBI_CHECK(cudaMemsetAsync(d, 0, sizeof(DSolve), ctx->stream));
              GBI_CHECK(cudaMemsetAsync(gp.cnt, 0, sizeof(unsigned int) * (S + 2), ctx->stream));
              if (hooks != nullptr) {
                GBI_TRY(hooks->before());
                GBI_TRY(pack_inputs());
              }
              GBI_TRY(rhs_pass());
              if (!warm) GBI_CHECK(cudaMemsetAsync(xQH, 0, sizeof(double) * nh, ctx->stream));
              {
                NormCtl nc{};
                nc.follow = kFollowRefine0;
                nc.rtol = rtol;
                bk_norm_then<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(b, N, h, B.off, gp, 2, nc);
                ++ctx->launches;
              }
              gk_guard<<<1, 256, 0, ctx->stream>>>(gp, P<unsigned int>(ctx->minr2), bad_in, s.a,
                                                   pairs_all > 0 ? prm->min_sep : 0.0, d);
              ++ctx->launches;
              if (!warm) {
                // sweep 0: the residual is b
                GBI_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * nh, cudaMemcpyDeviceToDevice, ctx->stream));
                GBI_CHECK(cudaMemsetAsync(dl, 0, sizeof(double) * nh, ctx->stream));
                GBI_TRY(emit_gmres(gb, s, B, gp, restart, r, dl, inner, max_iter, rtol, d));
                bk_axpy_enabled<<<g2, 256, 0, ctx->stream>>>(dl, N, B.sys, gp.st, xQH);
                ++ctx->launches;
              } else {
                // sweep 0 of a warm start (the guess packed before the graph): its residual
                // from an FP32 pass sizes the inner solve; the sweeps below check the result
                // in the high precision
                GBI_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * nh, cudaMemcpyDeviceToDevice, ctx->stream));
                PairArgs p = batched(pair_args(s, xQH, r, -1.0, 1.0, 1, s.ones, 6), nullptr);
                GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, 1, p));
                NormCtl nc{};
                nc.follow = kFollowWarm;
                nc.rtol = rtol;
                bk_norm_then<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(r, N, h, B.off, gp, 1, nc);
                ++ctx->launches;
                GBI_CHECK(cudaMemsetAsync(dl, 0, sizeof(double) * nh, ctx->stream));
                GBI_TRY(emit_gmres(gb, s, B, gp, restart, r, dl, inner, max_iter, rtol, d));
                bk_axpy_enabled<<<g2, 256, 0, ctx->stream>>>(dl, N, B.sys, gp.st, xQH);
                ++ctx->launches;
              }
              // sweeps 1, 2, ...: residual, refinement test, inner solve.  With updates (the
              // double-float modes) the first sweep's residual b - A_hp x is the only
              // high-precision pass; each inner solve's correction d then updates it as
              // r -= A_32 d (d is some 1e-6 of x, so FP32 adds ~1e-13 of |b|)
              if (incr) {
                gk_copy<<<grid1(nh), 256, 0, ctx->stream>>>(r, b, nh);
                ++ctx->launches;
                PairArgs p = batched(pair_args(s, xQH, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
                GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, hp, p));
              }
              const cudaGraphConditionalHandle hsw = gb.handle();
              gk_sweep_start<<<1, 256, 0, ctx->stream>>>(gp, hsw);
              ++ctx->launches;
              GBI_TRY(gb.body(gb.node(hsw, cudaGraphCondTypeWhile), kBodySweep, [&]() -> gbi_status {
                if (!incr) {
                  gk_copy<<<grid1(nh), 256, 0, ctx->stream>>>(r, b, nh);
                  ++ctx->launches;
                  PairArgs p = batched(pair_args(s, xQH, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
                  GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, hp, p));
                }
                const cudaGraphConditionalHandle hif = gb.handle();
                {
                  NormCtl nc{};
                  nc.follow = kFollowSweep;
                  nc.rtol = rtol;
                  nc.d = d;
                  nc.hsw = hsw;
                  nc.hif = hif;
                  nc.max_refine = max_refine;
                  nc.max_iter = max_iter;
                  nc.incr = incr ? 1 : 0;
                  bk_norm_then<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(r, N, h, B.off, gp, 1, nc);
                  ++ctx->launches;
                }
                GBI_CHECK(cudaGetLastError());
                return gb.body(gb.node(hif, cudaGraphCondTypeIf), kBodyIf, [&]() -> gbi_status {
                  gk_zero<<<grid1(nh), 256, 0, ctx->stream>>>(dl, nh);
                  ++ctx->launches;
                  GBI_TRY(emit_gmres(gb, s, B, gp, restart, r, dl, inner, max_iter, rtol, d));
                  bk_axpy_enabled<<<g2, 256, 0, ctx->stream>>>(dl, N, B.sys, gp.st, xQH);
                  ++ctx->launches;
                  if (incr) {
                    PairArgs p = batched(pair_args(s, dl, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
                    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, 1, p));
                  }
                  GBI_CHECK(cudaGetLastError());
                  return GBI_OK;
                });
              }));
              gk_summary<<<1, 256, 0, ctx->stream>>>(gp, d);
              ++ctx->launches;
              GBI_TRY(output_pass());
              if (hooks != nullptr) {
                GBI_TRY(unpack_outputs());
                GBI_TRY(hooks->after(d));
              }
              return GBI_OK;
            }();
            const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
            if (st == GBI_OK && (e != cudaSuccess || gb.err != cudaSuccess)) st = GBI_ERR_CUDA;
          }
          const long long total = ctx->launches - saved;
          ctx->launches = saved;
          if (st == GBI_OK && cudaGraphInstantiate(&ctx->solve_exec, graph, 0) != cudaSuccess) {
            ctx->solve_exec = nullptr;
            st = GBI_ERR_CUDA;
          }
          if (graph) cudaGraphDestroy(graph);
          if (st == GBI_OK) {
            built = true;
            ctx->solve_key = key;
            ctx->solve_prev = key;
            ctx->solve_own[0] = total - gb.nested[0];
            for (int i = 0; i < 4; ++i) ctx->solve_own[1 + i] = gb.own[i];
          }
        }
      }
      if (!built) {
        // the graph could not be built here: the host-driven sequence serves this key
        cudaGetLastError();
        ctx->solve_failed = key;
      }
    }
    if (ctx->solve_exec != nullptr && key == ctx->solve_key) {
      DSolve* d = P<DSolve>(ctx->dsolve);
      if (hooks == nullptr) {
        GBI_TRY(pack_inputs());
        if (warm) {
          k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, QH, hscale, 1.0, xQH, bad_in);
          ++ctx->launches;
          GBI_CHECK(cudaGetLastError());
        }
      }
      GBI_CHECK(cudaGraphLaunch(ctx->solve_exec, ctx->stream));
      ++ctx->solve_replays;
      if (hooks == nullptr) GBI_TRY(unpack_outputs());
      GBI_CHECK(cudaMemcpyAsync(hrec, d, sizeof(DSolve), cudaMemcpyDeviceToHost, ctx->stream));
      GBI_CHECK(cudaMemcpyAsync(hbits, ctx->minr2.p, 3 * sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
      GBI_CHECK(cudaStreamSynchronize(ctx->stream));
      if (hbits[1] != 0) {
        GBI_TRY(pass_error_reset(ctx));
        return GBI_ERR_TIMEOUT;
      }
      if (hbits[2] != 0 || hrec->bad_input) return GBI_ERR_ARG;
      const DSolve& hd = *hrec;
      ctx->launches += ctx->solve_own[0] + (long long)hd.refinements * ctx->solve_own[1] +
                       (long long)hd.ifs * ctx->solve_own[2] + hd.cycles * ctx->solve_own[3] +
                       hd.steps * ctx->solve_own[4];
      // the right-hand-side and output passes are the two the host knows of
      inf->iters = (int)hd.iters;
      inf->refinements = hd.refinements;
      inf->matvecs_f32 = (int)hd.mv32 + (io == 1 ? 2 : 0) + (warm ? 1 : 0);
      inf->matvecs_f64 = (int)hd.mv64 + (io == 1 ? 0 : 2);
      inf->pair_interactions = hd.pairs + (2 + (warm ? 1 : 0)) * pairs_all;
      inf->rel_residual = hd.rel_max;
      float mr2;
      std::memcpy(&mr2, hbits, sizeof(float));
      inf->min_separation = pairs_all > 0 ? std::sqrt(double(mr2)) / s.a : 0.0;
      if (hd.overlap) return GBI_ERR_OVERLAP;
      return hd.rel_max <= rtol ? GBI_OK : GBI_ERR_NOT_CONVERGED;
    }
  }

  if (hooks != nullptr) GBI_TRY(hooks->before());
  GBI_TRY(pack_inputs());
  GBI_TRY(rhs_pass());
  (io == 1 ? inf->matvecs_f32 : inf->matvecs_f64) += 1;
  inf->pair_interactions += pairs_all;
  {
    // inputs checked (and, with the guard on, the smallest distance) before the GMRES
    unsigned int bits[3] = {0, 0, 0};
    GBI_CHECK(cudaMemcpyAsync(bits, ctx->minr2.p, 3 * sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    if (bits[1] != 0) {
      GBI_TRY(pass_error_reset(ctx));
      return GBI_ERR_TIMEOUT;
    }
    if (bits[2] != 0) return GBI_ERR_ARG;
  }
  if (prm->min_sep > 0) {
    unsigned int bits[2] = {0, 0};
    GBI_CHECK(cudaMemcpyAsync(bits, ctx->minr2.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    float mr2;
    std::memcpy(&mr2, &bits[0], sizeof(float));
    inf->min_separation = pairs_all > 0 ? std::sqrt(double(mr2)) / s.a : 0.0;
    if (pairs_all > 0 && inf->min_separation < prm->min_sep) return GBI_ERR_OVERLAP;
  }

  // initial guess
  bool zero = true;
  if (warm_start) {
    k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, QH, hscale, 1.0, xQH, bad_in);
    ++ctx->launches;
    zero = false;
  } else {
    GBI_CHECK(cudaMemsetAsync(xQH, 0, sizeof(double) * nh, ctx->stream));
  }
  // |b_s| per system
  GBI_CHECK(cudaMemsetAsync(gp.cnt, 0, sizeof(unsigned int) * (S + 2), ctx->stream));
  auto norm_refine = [&](const double* x, int mode, int follow) {
    NormCtl nc{};
    nc.follow = follow;
    nc.rtol = rtol;
    bk_norm_then<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(x, N, h, B.off, gp, mode, nc);
    ++ctx->launches;
  };
  norm_refine(b, 2, kFollowRefine0);
  auto read_state = [&]() -> gbi_status {
    GBI_CHECK(cudaMemcpyAsync(hst, gp.st, sizeof(GDev) * S, cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    return GBI_OK;
  };
  auto pairs_enabled = [&]() {
    long long c = 0;
    for (int q = 0; q < S; ++q)
      if (hst[q].enabled) {
        const long long ns = B.h_off[q + 1] - B.h_off[q];
        c += ns * (ns - 1);
      }
    return c;
  };
  GBI_TRY(read_state());
  bool converged = false;
  if (prm->precision == 0) {
    int it = 0;
    double rr = 0.0;
    GBI_TRY(gmres_batch(ctx, s, B, 0, b, xQH, zero, rtol, restart, max_iter, inf, it, rr, hst, hbefore, hbar));
    inf->iters += it;
    // true FP64 residual per system
    GBI_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * nh, cudaMemcpyDeviceToDevice, ctx->stream));
    PairArgs p = batched(pair_args(s, xQH, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, 0, p));
    inf->matvecs_f64 += 1;
    inf->pair_interactions += pairs_enabled();
    norm_refine(r, 1, kFollowRefine1);
    GBI_TRY(read_state());
  } else {
    // mixed precision: r = b - A_hp x; A_32 d = r (FP32 pair sums, FP64 Arnoldi); x += d
    for (int sweep = 0;; ++sweep) {
      if (incr && sweep >= 2) {
        // the previous inner solve's correction updates the residual: r -= A_32 d
        PairArgs p = batched(pair_args(s, dl, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
        GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, 1, p));
        inf->matvecs_f32 += 1;
        inf->pair_interactions += pairs_enabled();
        norm_refine(r, 1, kFollowRefine1);
      } else {
        GBI_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * nh, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      if (!(zero && sweep == 0) && !(incr && sweep >= 2)) {
        // sweep 0 of a warm start: the guess's residual from an FP32 pass, which only
        // sizes the inner solve (the later sweeps check in the high precision)
        const bool warm0 = !zero && sweep == 0;
        PairArgs p = batched(pair_args(s, xQH, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
        GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, warm0 ? 1 : hp, p));
        (warm0 ? inf->matvecs_f32 : inf->matvecs_f64) += 1;
        inf->pair_interactions += pairs_enabled();
        norm_refine(r, 1, warm0 ? kFollowWarm : kFollowRefine1);
      }
      if (sweep > 0) inf->refinements += 1;
      if (sweep >= max_refine || inf->iters >= max_iter) {
        GBI_TRY(read_state());
        break;
      }
      int it = 0;
      double rr = 0.0;
      GBI_CHECK(cudaMemsetAsync(dl, 0, sizeof(double) * nh, ctx->stream));
      GBI_TRY(gmres_batch(ctx, s, B, 1, r, dl, true, inner, restart, max_iter - inf->iters, inf, it, rr, hst, hbefore, hbar,
                          rtol));
      inf->iters += it;
      bool any = false;
      for (int q = 0; q < S; ++q) any = any || hst[q].enabled;
      if (!any) break;       // every system met the tolerance at this sweep's residual
      bk_axpy_enabled<<<g2, 256, 0, ctx->stream>>>(dl, N, B.sys, gp.st, xQH);
      ++ctx->launches;
      GBI_CHECK(cudaGetLastError());
    }
  }
  converged = true;
  inf->rel_residual = 0.0;
  for (int q = 0; q < S; ++q) {
    inf->rel_residual = std::max(inf->rel_residual, hst[q].rel);
    if (hst[q].rel > rtol) converged = false;
  }
  GBI_TRY(output_pass());
  GBI_TRY(unpack_outputs());
  if (converged && hooks != nullptr) GBI_TRY(hooks->after(nullptr));
  (io == 1 ? inf->matvecs_f32 : inf->matvecs_f64) += 1;
  inf->pair_interactions += pairs_all;
  unsigned int bits[3] = {0, 0, 0};
  GBI_CHECK(cudaMemcpyAsync(bits, ctx->minr2.p, 3 * sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  if (bits[1] != 0) {
    GBI_TRY(pass_error_reset(ctx));
    return GBI_ERR_TIMEOUT;
  }
  if (bits[2] != 0) return GBI_ERR_ARG;
  if (prm->min_sep <= 0) {
    float mr2;
    std::memcpy(&mr2, &bits[0], sizeof(float));
    inf->min_separation = pairs_all > 0 ? std::sqrt(double(mr2)) / s.a : 0.0;
  }
  return converged ? GBI_OK : GBI_ERR_NOT_CONVERGED;
}

}  // namespace gbi
