// Learned near-field correction: neighbour lists, pair features, the tanh network
// (BF16 tensor-core inference, FP32 training with the inference's BF16 rounding),
// per-sphere sums and Adam.
//
// The network corrects the superposition velocities of Sec. IV toward the Galerkin
// solution of Sec. II-III for every ordered pair closer than rcut * a (the paper has
// no network; this is an engineering addition).  Pair frame, features, layer sizes
// and the flat parameter layout are stated in include/gbi.h next to gbi_mlp_set.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbi_internal.cuh"

namespace gbi {
namespace mlpk {

constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH * NH;
constexpr int OFF_W4 = OFF_B3 + NH;
constexpr int OFF_B4 = OFF_W4 + NOUT * NH;
static_assert(OFF_B4 + NOUT == NPARAM, "parameter layout");

// ---------------------------------------------------------------------------------
// exclusive scan of int counts (chunks of 1024, one level of chunk sums: n <= 2^20)
// ---------------------------------------------------------------------------------

__device__ __forceinline__ int block_exclusive_scan_1024(int v, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_warp[lane] = t;   // inclusive warp totals
  }
  __syncthreads();
  total = s_warp[31];
  const int before = w > 0 ? s_warp[w - 1] : 0;
  return before + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_chunks(const int* __restrict__ in, int* __restrict__ out, int n,
                                                      int* __restrict__ sums) {
  __shared__ int s_warp[32];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  int total = 0;
  const int e = block_exclusive_scan_1024(v, s_warp, total);
  if (i < n) out[i] = e;
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int* __restrict__ sums, int nchunks, int* __restrict__ total_out) {
  __shared__ int s_warp[32];
  const int v = threadIdx.x < nchunks ? sums[threadIdx.x] : 0;
  int total = 0;
  const int e = block_exclusive_scan_1024(v, s_warp, total);
  if (threadIdx.x < nchunks) sums[threadIdx.x] = e;
  if (threadIdx.x == 0) *total_out = total;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ sums) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n && blockIdx.x > 0) out[i] += sums[blockIdx.x];
}

size_t scan_scratch_ints(int n) { return (size_t)((n + 1023) / 1024) + 1; }

cudaError_t exclusive_scan(const int* in, int* out, int n, int* scratch, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int chunks = (n + 1023) / 1024;
  if (chunks > 1024) return cudaErrorInvalidValue;
  k_scan_chunks<<<chunks, 1024, 0, st>>>(in, out, n, scratch);
  k_scan_sums<<<1, 1024, 0, st>>>(scratch, chunks, scratch + chunks);
  k_scan_add<<<chunks, 1024, 0, st>>>(out, n, scratch);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// neighbour lists: ordered pairs (n, m), m != n, same system, |R_n - R_m| < rcut a,
// grouped by n and sorted by m within a group (so sums over them have a fixed order)
// ---------------------------------------------------------------------------------

// r^2 with the operation order of (dx dx + dy dy) + dz dz and no contraction, so that
// the inclusion test is the same as a plain FP64 evaluation on the host
__device__ __forceinline__ double dist2(const double* a, const double* b) {
  const double dx = __dsub_rn(a[0], b[0]), dy = __dsub_rn(a[1], b[1]), dz = __dsub_rn(a[2], b[2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// small systems (or one system small enough for O(N^2)): scan the whole system
__global__ void k_nb_sys(int N, const double* __restrict__ R, const int* __restrict__ sys_of,
                         const int* __restrict__ sys_off, double rc2, const int* __restrict__ start,
                         int* __restrict__ cnt, int* __restrict__ tg, int* __restrict__ sr) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  int lo = 0, hi = N;
  if (sys_of != nullptr) {
    lo = sys_off[sys_of[n]];
    hi = sys_off[sys_of[n] + 1];
  }
  const double* rn = R + 3 * (size_t)n;
  int c = 0;
  const int base = start != nullptr ? start[n] : 0;
  for (int m = lo; m < hi; ++m) {
    if (m == n) continue;
    if (dist2(rn, R + 3 * (size_t)m) < rc2) {
      if (start != nullptr) {
        tg[base + c] = n;
        sr[base + c] = m;
      }
      ++c;
    }
  }
  if (start == nullptr) cnt[n] = c;
}

struct CellGrid {
  double lo[3];
  double inv;      // 1 / cell side
  int dim[3];
};

__device__ __forceinline__ int cell_coord(double x, double lo, double inv, int dim) {
  int c = int(floor((x - lo) * inv));
  return c < 0 ? 0 : (c >= dim ? dim - 1 : c);
}

__global__ void k_cell_count(int N, const double* __restrict__ R, CellGrid g, int* __restrict__ cell_of,
                             int* __restrict__ cell_cnt) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double* r = R + 3 * (size_t)n;
  const int cx = cell_coord(r[0], g.lo[0], g.inv, g.dim[0]);
  const int cy = cell_coord(r[1], g.lo[1], g.inv, g.dim[1]);
  const int cz = cell_coord(r[2], g.lo[2], g.inv, g.dim[2]);
  const int c = (cz * g.dim[1] + cy) * g.dim[0] + cx;
  cell_of[n] = c;
  atomicAdd(&cell_cnt[c], 1);
}

// slot order within a cell depends on timing; the neighbour lists are sorted afterwards
__global__ void k_cell_fill(int N, const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                            int* __restrict__ cell_fill, int* __restrict__ items) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int c = cell_of[n];
  items[cell_start[c] + atomicAdd(&cell_fill[c], 1)] = n;
}

constexpr int kMaxNb = 64;   // neighbours kept per sphere in the cell-list path

__global__ void k_nb_cells(int N, const double* __restrict__ R, CellGrid g, const int* __restrict__ cell_of,
                           const int* __restrict__ cell_start, const int* __restrict__ cell_cnt,
                           const int* __restrict__ items, double rc2, const int* __restrict__ start,
                           int* __restrict__ cnt, int* __restrict__ tg, int* __restrict__ sr,
                           int* __restrict__ overflow) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double* rn = R + 3 * (size_t)n;
  const int c = cell_of[n];
  const int cx = c % g.dim[0], cy = (c / g.dim[0]) % g.dim[1], cz = c / (g.dim[0] * g.dim[1]);
  int nb[kMaxNb];
  int k = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= g.dim[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = cy + dy;
      if (y < 0 || y >= g.dim[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = cx + dx;
        if (x < 0 || x >= g.dim[0]) continue;
        const int cc = (z * g.dim[1] + y) * g.dim[0] + x;
        const int b = cell_start[cc], e = b + cell_cnt[cc];
        for (int i = b; i < e; ++i) {
          const int m = items[i];
          if (m == n || !(dist2(rn, R + 3 * (size_t)m) < rc2)) continue;
          if (k < kMaxNb) nb[k] = m;
          ++k;
        }
      }
    }
  }
  if (k > kMaxNb) {
    atomicExch(overflow, 1);
    k = kMaxNb;
  }
  if (start == nullptr) {
    cnt[n] = k;
    return;
  }
  // insertion sort by source index: the list no longer depends on the cell slot order
  for (int i = 1; i < k; ++i) {
    const int v = nb[i];
    int j = i - 1;
    while (j >= 0 && nb[j] > v) {
      nb[j + 1] = nb[j];
      --j;
    }
    nb[j + 1] = v;
  }
  const int base = start[n];
  for (int i = 0; i < k; ++i) {
    tg[base + i] = n;
    sr[base + i] = nb[i];
  }
}

__global__ void k_bbox(int N, const double* __restrict__ R, double* __restrict__ part) {
  __shared__ double s[6][256];
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) {
      mn[d] = fmin(mn[d], R[3 * (size_t)n + d]);
      mx[d] = fmax(mx[d], R[3 * (size_t)n + d]);
    }
  for (int d = 0; d < 3; ++d) {
    s[d][threadIdx.x] = mn[d];
    s[3 + d][threadIdx.x] = mx[d];
  }
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + o]);
        s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + o]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// ---------------------------------------------------------------------------------
// pair features (FP32 after an FP64 difference of the centres)
// ---------------------------------------------------------------------------------

__global__ void k_features(int P, const double* __restrict__ R, const double* __restrict__ p,
                           const int* __restrict__ tg, const int* __restrict__ sr, double a,
                           float* __restrict__ F, float* __restrict__ FR) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const int n = tg[k], m = sr[k];
  const float rx = float(R[3 * (size_t)n] - R[3 * (size_t)m]);
  const float ry = float(R[3 * (size_t)n + 1] - R[3 * (size_t)m + 1]);
  const float rz = float(R[3 * (size_t)n + 2] - R[3 * (size_t)m + 2]);
  const float pn[3] = {float(p[3 * (size_t)n]), float(p[3 * (size_t)n + 1]), float(p[3 * (size_t)n + 2])};
  const float pm[3] = {float(p[3 * (size_t)m]), float(p[3 * (size_t)m + 1]), float(p[3 * (size_t)m + 2])};
  const float r = sqrtf(rx * rx + ry * ry + rz * rz);
  const float ez[3] = {rx / r, ry / r, rz / r};
  float t[3];
  float c = pn[0] * ez[0] + pn[1] * ez[1] + pn[2] * ez[2];
  for (int i = 0; i < 3; ++i) t[i] = pn[i] - c * ez[i];
  float t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  if (t2 <= 1e-12f) {
    c = pm[0] * ez[0] + pm[1] * ez[1] + pm[2] * ez[2];
    for (int i = 0; i < 3; ++i) t[i] = pm[i] - c * ez[i];
    t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  }
  if (t2 <= 1e-12f) {
    int ax = 0;
    if (fabsf(ez[1]) < fabsf(ez[ax])) ax = 1;
    if (fabsf(ez[2]) < fabsf(ez[ax])) ax = 2;
    for (int i = 0; i < 3; ++i) t[i] = (i == ax ? 1.f : 0.f) - ez[ax] * ez[i];
    t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  }
  const float inv = 1.0f / sqrtf(t2);
  const float ex[3] = {t[0] * inv, t[1] * inv, t[2] * inv};
  const float ey[3] = {ez[1] * ex[2] - ez[2] * ex[1], ez[2] * ex[0] - ez[0] * ex[2], ez[0] * ex[1] - ez[1] * ex[0]};
  const float u = float(2.0 * a) / r;
  const float d = fmaxf(r / float(a) - 2.0f, 0.01f);
  float* f = F + (size_t)k * NIN;
  f[0] = u;
  f[1] = u * u * u;
  f[2] = d;
  f[3] = logf(d);
  f[4] = pn[0] * ez[0] + pn[1] * ez[1] + pn[2] * ez[2];
  f[5] = pn[0] * ex[0] + pn[1] * ex[1] + pn[2] * ex[2];
  f[6] = pm[0] * ex[0] + pm[1] * ex[1] + pm[2] * ex[2];
  f[7] = pm[0] * ey[0] + pm[1] * ey[1] + pm[2] * ey[2];
  f[8] = pm[0] * ez[0] + pm[1] * ez[1] + pm[2] * ez[2];
  float* fr = FR + (size_t)k * 9;
  for (int i = 0; i < 3; ++i) {
    fr[i] = ex[i];
    fr[3 + i] = ey[i];
    fr[6 + i] = ez[i];
  }
}

// ---------------------------------------------------------------------------------
// weights: bf16-rounded FP32 copy (training forward) and padded bf16 copy (inference)
// ---------------------------------------------------------------------------------

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// padded inference layout: W1 [128][K1P], W2 [128][LDW], W3 [128][LDW], W4 [8][LDW] (bf16),
// then b1, b2, b3 [128], b4 [8] (FP32)
constexpr int K1P = 24;    // layer-1 rows: 9 inputs, zero-padded; 48-byte rows
constexpr int LDW = 136;   // 128-wide rows padded to 272 bytes (conflict-free ldmatrix)
constexpr int PK_W1 = 0;
constexpr int PK_W2 = PK_W1 + NH * K1P;
constexpr int PK_W3 = PK_W2 + NH * LDW;
constexpr int PK_W4 = PK_W3 + NH * LDW;
constexpr int PK_END = PK_W4 + 8 * LDW;          // bf16 elements
constexpr int PK_BIAS_FLOATS = 3 * NH + 8;
size_t packed_bytes() { return sizeof(__nv_bfloat16) * PK_END + sizeof(float) * PK_BIAS_FLOATS; }

__device__ __forceinline__ bool is_bias(int i) {
  return (i >= OFF_B1 && i < OFF_B1 + NH) || (i >= OFF_B2 && i < OFF_B2 + NH) || (i >= OFF_B3 && i < OFF_B3 + NH) ||
         i >= OFF_B4;
}

// thq: weights rounded to bf16 (what the tensor cores multiply), biases kept in FP32
__global__ void k_pack(const float* __restrict__ th, float* __restrict__ thq, __nv_bfloat16* __restrict__ pk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NPARAM) thq[i] = is_bias(i) ? th[i] : bf16r(th[i]);
  float* bias = reinterpret_cast<float*>(pk + PK_END);
  if (i < NH * K1P) {
    const int j = i / K1P, k = i % K1P;
    pk[PK_W1 + i] = __float2bfloat16_rn(k < NIN ? th[OFF_W1 + j * NIN + k] : 0.f);
  }
  if (i < NH * LDW) {
    const int j = i / LDW, k = i % LDW;
    pk[PK_W2 + i] = __float2bfloat16_rn(k < NH ? th[OFF_W2 + j * NH + k] : 0.f);
    pk[PK_W3 + i] = __float2bfloat16_rn(k < NH ? th[OFF_W3 + j * NH + k] : 0.f);
  }
  if (i < 8 * LDW) {
    const int j = i / LDW, k = i % LDW;
    pk[PK_W4 + i] = __float2bfloat16_rn((j < NOUT && k < NH) ? th[OFF_W4 + j * NH + k] : 0.f);
  }
  if (i < NH) {
    bias[i] = th[OFF_B1 + i];
    bias[NH + i] = th[OFF_B2 + i];
    bias[2 * NH + i] = th[OFF_B3 + i];
  }
  if (i < 8) bias[3 * NH + i] = i < NOUT ? th[OFF_B4 + i] : 0.f;
}

cudaError_t pack_weights(const float* theta, float* thq, void* packed, cudaStream_t st) {
  k_pack<<<(NPARAM + 255) / 256, 256, 0, st>>>(theta, thq, static_cast<__nv_bfloat16*>(packed));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// inference: BF16 tensor-core MMA (m16n8k16, FP32 accumulate), 64 pairs per tile,
// four warps of 16 pairs each, weights resident in shared memory, persistent blocks
// ---------------------------------------------------------------------------------

constexpr int TILE_P = 64;
constexpr int LDA = 136;   // activation rows (bf16)
constexpr int LDF = 24;    // feature rows (bf16)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// one hidden layer for the warp's 16 rows: act[16 x 128] (bf16, in place) <- tanh(A W^T + b)
// where A is read from `in` (row stride lda, K columns) and W from shared memory
template <int K, int LDIN, int LDWT>
__device__ __forceinline__ void hidden_layer(const __nv_bfloat16* in, const __nv_bfloat16* W, const float* b,
                                             __nv_bfloat16* out, int lane) {
  float acc[16][4];
#pragma unroll
  for (int t = 0; t < 16; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    uint32_t a0, a1, a2, a3;
    ldsm_x4(smem_u32(in + (lane & 15) * LDIN + ks * 16 + (lane >> 4) * 8), a0, a1, a2, a3);
#pragma unroll
    for (int t2 = 0; t2 < 8; ++t2) {
      // two n-tiles (16 outputs) per ldmatrix.x4 of W rows
      const int row = t2 * 16 + (lane & 7) + ((lane >> 4) << 3);
      const int col = ks * 16 + ((lane >> 3) & 1) * 8;
      uint32_t b0, b1, b2, b3;
      ldsm_x4(smem_u32(W + row * LDWT + col), b0, b1, b2, b3);
      mma_bf16(acc[2 * t2], a0, a1, a2, a3, b0, b1);
      mma_bf16(acc[2 * t2 + 1], a0, a1, a2, a3, b2, b3);
    }
  }
  __syncwarp();
  const int g = lane >> 2, c2 = (lane & 3) * 2;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int col = t * 8 + c2;
    const float v0 = tanh_act(acc[t][0] + b[col]), v1 = tanh_act(acc[t][1] + b[col + 1]);
    const float v2 = tanh_act(acc[t][2] + b[col]), v3 = tanh_act(acc[t][3] + b[col + 1]);
    *reinterpret_cast<uint32_t*>(out + g * LDA + col) = pack_bf16x2(v0, v1);
    *reinterpret_cast<uint32_t*>(out + (g + 8) * LDA + col) = pack_bf16x2(v2, v3);
  }
  __syncwarp();
}

__global__ void __launch_bounds__(128) k_infer(int P, const float* __restrict__ F, const float* __restrict__ FR,
                                                const __nv_bfloat16* __restrict__ pk, float* __restrict__ out,
                                                int head) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem_raw);                 // PK_END
  float* sB = reinterpret_cast<float*>(sW + PK_END);                                // biases
  __nv_bfloat16* sF = reinterpret_cast<__nv_bfloat16*>(sB + PK_BIAS_FLOATS);       // [64][LDF]
  __nv_bfloat16* sA = sF + TILE_P * LDF;                                            // [64][LDA]
  float* sO = reinterpret_cast<float*>(sA + TILE_P * LDA);                          // [64][8]

  // weights and biases once per block (16-byte copies)
  {
    const int4* src = reinterpret_cast<const int4*>(pk);
    int4* dst = reinterpret_cast<int4*>(smem_raw);
    const int n16 = int((sizeof(__nv_bfloat16) * PK_END + sizeof(float) * PK_BIAS_FLOATS) / 16);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (P + TILE_P - 1) / TILE_P;
  __nv_bfloat16* fw = sF + warp * 16 * LDF;
  __nv_bfloat16* aw = sA + warp * 16 * LDA;
  float* ow = sO + warp * 16 * 8;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int p0 = tile * TILE_P + warp * 16;
    // features of the warp's 16 pairs -> bf16, zero-padded to 16 columns
    for (int i = lane; i < 16 * 16; i += 32) {
      const int r = i >> 4, k = i & 15;
      const int pp = p0 + r;
      const float v = (k < NIN && pp < P) ? F[(size_t)pp * NIN + k] : 0.f;
      fw[r * LDF + k] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    hidden_layer<16, LDF, K1P>(fw, sW + PK_W1, sB, aw, lane);
    hidden_layer<128, LDA, LDW>(aw, sW + PK_W2, sB + NH, aw, lane);
    hidden_layer<128, LDA, LDW>(aw, sW + PK_W3, sB + 2 * NH, aw, lane);
    // output layer: 8 columns (6 used), one n-tile
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
      uint32_t a0, a1, a2, a3, b0, b1;
      ldsm_x4(smem_u32(aw + (lane & 15) * LDA + ks * 16 + (lane >> 4) * 8), a0, a1, a2, a3);
      ldsm_x2(smem_u32(sW + PK_W4 + (lane & 7) * LDW + ks * 16 + ((lane >> 3) & 1) * 8), b0, b1);
      mma_bf16(acc, a0, a1, a2, a3, b0, b1);
    }
    {
      const int g = lane >> 2, c2 = (lane & 3) * 2;
      const float* b4 = sB + 3 * NH;
      ow[g * 8 + c2] = acc[0] + b4[c2];
      ow[g * 8 + c2 + 1] = acc[1] + b4[c2 + 1];
      ow[(g + 8) * 8 + c2] = acc[2] + b4[c2];
      ow[(g + 8) * 8 + c2 + 1] = acc[3] + b4[c2 + 1];
    }
    __syncwarp();
    if (lane < 16) {
      const int pp = p0 + lane;
      if (pp < P) {
        const float* o = ow + lane * 8;
        float* dst = out + (size_t)pp * NOUT;
        if (FR != nullptr) {
          pair_out_to_lab(head, FR + (size_t)pp * 9, o, dst);   // frame rows e_x, e_y, e_z
        } else {
#pragma unroll
          for (int c = 0; c < NOUT; ++c) dst[c] = o[c];
        }
      }
    }
    __syncwarp();
  }
}

size_t infer_smem_bytes() {
  return sizeof(__nv_bfloat16) * PK_END + sizeof(float) * PK_BIAS_FLOATS +
         sizeof(__nv_bfloat16) * TILE_P * (LDF + LDA) + sizeof(float) * TILE_P * 8;
}

cudaError_t infer(int P, const float* F, const float* FR, const void* packed, float* out, int num_sms, int head,
                  cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  const size_t smem = infer_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int ntiles = (P + TILE_P - 1) / TILE_P;
  const int grid = ntiles < 2 * num_sms ? ntiles : 2 * num_sms;
  k_infer<<<grid, 128, smem, st>>>(P, F, FR, static_cast<const __nv_bfloat16*>(packed), out, head);
  return cudaGetLastError();
}

// per-sphere fixed-order sums of the rotated pair outputs, scaled and added to V, Omega
__global__ void k_sphere_sums(int N, const int* __restrict__ start, const float* __restrict__ lab, double scale,
                              double* __restrict__ V, double* __restrict__ Om) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int k = start[n]; k < start[n + 1]; ++k)
    for (int c = 0; c < 6; ++c) s[c] += double(lab[(size_t)k * 6 + c]);
  for (int i = 0; i < 3; ++i) {
    V[3 * (size_t)n + i] += scale * s[i];
    Om[3 * (size_t)n + i] += scale * s[3 + i];
  }
}

cudaError_t sphere_sums(int N, const int* start, const float* lab, double scale, double* V, double* Om,
                        cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  k_sphere_sums<<<(N + 127) / 128, 128, 0, st>>>(N, start, lab, scale, V, Om);
  return cudaGetLastError();
}

// the same for the strain-mode head: the first five outputs into the 2s block of Q^H
__global__ void k_sphere_sums_q(int N, const int* __restrict__ start, const float* __restrict__ lab, double scale,
                                double* __restrict__ QH, int h) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s[5] = {0, 0, 0, 0, 0};
  for (int k = start[n]; k < start[n + 1]; ++k)
    for (int c = 0; c < 5; ++c) s[c] += double(lab[(size_t)k * 6 + c]);
  for (int c = 0; c < 5; ++c) QH[(size_t)h * n + c] += scale * s[c];
}

cudaError_t sphere_sums_q(int N, const int* start, const float* lab, double scale, double* QH, int h,
                          cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  k_sphere_sums_q<<<(N + 127) / 128, 128, 0, st>>>(N, start, lab, scale, QH, h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// training on the FP32 CUDA cores (engine 0; engine 1 trains on the tensor cores, the
// backward kernel in mlp_tc.cu): the forward pass multiplies the same bf16-rounded
// weights and layer inputs as the tensor-core inference; gradients flow straight
// through the rounding.  TP pairs per block, one thread per neuron.  Every tile writes a
// full partial gradient, so smaller tiles (more blocks per batch) cost more in those writes
// and their reduction than they gain in occupancy (measured: 8-pair tiles trained 23 %
// slower than 32-pair tiles).
// ---------------------------------------------------------------------------------

constexpr int TP = 32;

struct TrainSmem {
  float x0[TP][NIN];
  float h[3][TP][NH];      // tanh outputs (unrounded)
  float hq[3][TP][NH];     // bf16-rounded copies (the next layer's inputs)
  float o[TP][8];
};

__device__ void train_forward_tile(const float* __restrict__ thq, const float* __restrict__ F, int p0, int np,
                                   TrainSmem& s) {
  const int j = threadIdx.x;   // neuron
  for (int i = threadIdx.x; i < TP * NIN; i += blockDim.x) {
    const int r = i / NIN, k = i % NIN;
    s.x0[r][k] = r < np ? bf16r(F[(size_t)(p0 + r) * NIN + k]) : 0.f;
  }
  __syncthreads();
  {
    float w[NIN];
    for (int k = 0; k < NIN; ++k) w[k] = thq[OFF_W1 + j * NIN + k];
    const float bj = thq[OFF_B1 + j];
    for (int r = 0; r < TP; ++r) {
      float z = 0.f;
      for (int k = 0; k < NIN; ++k) z = fmaf(w[k], s.x0[r][k], z);
      const float t = tanhf(z + bj);
      s.h[0][r][j] = t;
      s.hq[0][r][j] = bf16r(t);
    }
  }
  __syncthreads();
  for (int L = 1; L < 3; ++L) {
    const float* W = thq + (L == 1 ? OFF_W2 : OFF_W3) + j * NH;
    const float bj = thq[(L == 1 ? OFF_B2 : OFF_B3) + j];
    float z[TP];
    for (int r = 0; r < TP; ++r) z[r] = 0.f;
    for (int k = 0; k < NH; ++k) {
      const float w = W[k];
      for (int r = 0; r < TP; ++r) z[r] = fmaf(w, s.hq[L - 1][r][k], z[r]);
    }
    for (int r = 0; r < TP; ++r) {
      const float t = tanhf(z[r] + bj);
      s.h[L][r][j] = t;
      s.hq[L][r][j] = bf16r(t);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < TP * NOUT; i += blockDim.x) {
    const int r = i / NOUT, c = i % NOUT;
    float z = 0.f;
    for (int k = 0; k < NH; ++k) z = fmaf(thq[OFF_W4 + c * NH + k], s.hq[2][r][k], z);
    s.o[r][c] = z + thq[OFF_B4 + c];
  }
  __syncthreads();
}

// lab [P][6] = rotated outputs of the pairs [p_begin, p_end)
__global__ void __launch_bounds__(NH) k_train_forward(const float* __restrict__ thq, const float* __restrict__ F,
                                                      const float* __restrict__ FR, int p_begin, int p_end,
                                                      float* __restrict__ lab, int head) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int p0 = p_begin + blockIdx.x * TP;
  const int np = min(TP, p_end - p0);
  train_forward_tile(thq, F, p0, np, s);
  for (int r = threadIdx.x; r < np; r += blockDim.x)
    pair_out_to_lab(head, FR + (size_t)(p0 + r) * 9, s.o[r], lab + (size_t)(p0 + r) * 6);
}

// per sphere n of [n_begin, n_end): P_n = sum of its pairs' rotated outputs; loss term
// |P_n - L_n|^2 / (6 Ns); dO of each of its pairs = FR * dP_n.  Block partial losses.
__global__ void k_train_loss(int n_begin, int n_end, const int* __restrict__ start, const float* __restrict__ lab,
                             const float* __restrict__ FR, const double* __restrict__ labels, double inv6ns,
                             float* __restrict__ dO, double* __restrict__ loss_part, int head) {
  __shared__ double s[128];
  const int n = n_begin + blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (n < n_end) {
    double pr[6] = {0, 0, 0, 0, 0, 0};
    for (int k = start[n]; k < start[n + 1]; ++k)
      for (int c = 0; c < 6; ++c) pr[c] += double(lab[(size_t)k * 6 + c]);
    float dp[6];
    for (int c = 0; c < 6; ++c) {
      const double d = pr[c] - labels[(size_t)n * 6 + c];
      l += d * d;
      dp[c] = float(2.0 * d * inv6ns);
    }
    for (int k = start[n]; k < start[n + 1]; ++k) lab_grad_to_pair(head, FR + (size_t)k * 9, dp, dO + (size_t)k * 6);
  }
  s[threadIdx.x] = l * inv6ns;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = s[0];
}

// backward of one tile: partial gradient of the flat parameters -> part[blockIdx.x]
__global__ void __launch_bounds__(NH) k_train_backward(const float* __restrict__ thq, const float* __restrict__ F,
                                                       const float* __restrict__ dO, int p_begin, int p_end,
                                                       float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
  float (*dz)[NH] = reinterpret_cast<float (*)[NH]>(smem_raw + sizeof(TrainSmem));            // [TP][NH]
  float (*dz2)[NH] = reinterpret_cast<float (*)[NH]>(smem_raw + sizeof(TrainSmem) + sizeof(float) * TP * NH);
  __shared__ float s_do[TP][8];
  const int p0 = p_begin + blockIdx.x * TP;
  const int np = min(TP, p_end - p0);
  train_forward_tile(thq, F, p0, np, s);
  const int j = threadIdx.x;
  float* g = part + (size_t)blockIdx.x * NPARAM;
  for (int i = threadIdx.x; i < TP * 8; i += blockDim.x) {
    const int r = i / 8, c = i % 8;
    s_do[r][c] = (r < np && c < NOUT) ? dO[(size_t)(p0 + r) * 6 + c] : 0.f;
  }
  __syncthreads();
  // output layer: dW4[c][j] = sum_r dO[r][c] hq3[r][j]; dh3 = dO W4
  for (int c = 0; c < NOUT; ++c) {
    float acc = 0.f;
    for (int r = 0; r < TP; ++r) acc = fmaf(s_do[r][c], s.hq[2][r][j], acc);
    g[OFF_W4 + c * NH + j] = acc;
  }
  if (j < NOUT) {
    float acc = 0.f;
    for (int r = 0; r < TP; ++r) acc += s_do[r][j];
    g[OFF_B4 + j] = acc;
  }
  for (int r = 0; r < TP; ++r) {
    float acc = 0.f;
    for (int c = 0; c < NOUT; ++c) acc = fmaf(s_do[r][c], thq[OFF_W4 + c * NH + j], acc);
    const float h = s.h[2][r][j];
    dz[r][j] = acc * (1.f - h * h);
  }
  __syncthreads();
  // hidden layers 3 and 2: dW[j][k] = sum_r dz[r][j] hq_prev[r][k]; dh_prev[r][k] = sum_j dz[r][j] W[j][k]
  for (int L = 2; L >= 1; --L) {
    const int offW = L == 2 ? OFF_W3 : OFF_W2, offB = L == 2 ? OFF_B3 : OFF_B2;
    float (*cur)[NH] = (L == 2) ? dz : dz2;
    float (*nxt)[NH] = (L == 2) ? dz2 : dz;
    for (int k = 0; k < NH; ++k) {
      float acc = 0.f;
      for (int r = 0; r < TP; ++r) acc = fmaf(cur[r][j], s.hq[L - 1][r][k], acc);
      g[offW + j * NH + k] = acc;
    }
    {
      float acc = 0.f;
      for (int r = 0; r < TP; ++r) acc += cur[r][j];
      g[offB + j] = acc;
    }
    // thread j now computes column j of dh_prev: sum_i cur[r][i] W[i][j]
    float acc[TP];
    for (int r = 0; r < TP; ++r) acc[r] = 0.f;
    for (int i = 0; i < NH; ++i) {
      const float w = thq[offW + i * NH + j];
      for (int r = 0; r < TP; ++r) acc[r] = fmaf(cur[r][i], w, acc[r]);
    }
    for (int r = 0; r < TP; ++r) {
      const float h = s.h[L - 1][r][j];
      nxt[r][j] = acc[r] * (1.f - h * h);
    }
    __syncthreads();
  }
  // first layer: dz (from L = 1 above) holds dz1
  for (int k = 0; k < NIN; ++k) {
    float acc = 0.f;
    for (int r = 0; r < TP; ++r) acc = fmaf(dz[r][j], s.x0[r][k], acc);
    g[OFF_W1 + j * NIN + k] = acc;
  }
  {
    float acc = 0.f;
    for (int r = 0; r < TP; ++r) acc += dz[r][j];
    g[OFF_B1 + j] = acc;
  }
}

size_t train_smem_bytes() { return sizeof(TrainSmem) + 2 * sizeof(float) * TP * NH; }

// grad[i] = sum over tiles of part[t][i] in a fixed grouping: eight FP64 partial sums over
// t = k, k + 8, ... (short dependent chains; an FP64 add has ~64 cycles of latency on
// GB300), then added in k order
__global__ void k_grad_reduce(int ntiles, const float* __restrict__ part, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int t = 0;
  for (; t + 8 <= ntiles; t += 8) {
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += double(part[(size_t)(t + k) * NPARAM + i]);
  }
  for (int k = 0; t + k < ntiles; ++k) s[k] += double(part[(size_t)(t + k) * NPARAM + i]);
  double tot = s[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) tot += s[k];
  grad[i] = float(tot);
}

cudaError_t train_batch(const float* thq, const float* F, const float* FR, const int* start, const double* labels,
                        int p_begin, int p_end, int n_begin, int n_end, int ns_total, float* lab, float* dO,
                        float* part, double* loss_part, float* grad, int head, int engine, const void* packed_tc,
                        int* err, int num_sms, cudaStream_t st) {
  const int np = p_end - p_begin;
  const int nb = (n_end - n_begin + 127) / 128;
  if (engine == 1) {
    // tensor cores: the forward of the inference kernel, the loss, the backward kernel
    cudaError_t e = cudaSuccess;
    if (np > 0) e = infer_tc(np, F + (size_t)p_begin * NIN, FR + (size_t)p_begin * 9, packed_tc,
                             lab + (size_t)p_begin * 6, err, num_sms, head, st);
    if (e != cudaSuccess) return e;
    if (nb > 0)
      k_train_loss<<<nb, 128, 0, st>>>(n_begin, n_end, start, lab, FR, labels, 1.0 / (6.0 * ns_total), dO,
                                       loss_part, head);
    if (np > 0) {
      e = train_bwd_tc(np, F + (size_t)p_begin * NIN, dO + (size_t)p_begin * 6, packed_tc, part, err, num_sms, st);
      if (e != cudaSuccess) return e;
      k_grad_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(train_bwd_tc_blocks(np, num_sms), part, grad);
    } else {
      cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, st);
    }
    return cudaGetLastError();
  }
  const int ntiles = (np + TP - 1) / TP;
  const size_t smem_f = sizeof(TrainSmem), smem_b = train_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_train_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_f));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_train_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_b));
  if (e != cudaSuccess) return e;
  if (ntiles > 0) k_train_forward<<<ntiles, NH, smem_f, st>>>(thq, F, FR, p_begin, p_end, lab, head);
  if (nb > 0)
    k_train_loss<<<nb, 128, 0, st>>>(n_begin, n_end, start, lab, FR, labels, 1.0 / (6.0 * ns_total), dO,
                                     loss_part, head);
  if (ntiles > 0) {
    k_train_backward<<<ntiles, NH, smem_b, st>>>(thq, F, dO, p_begin, p_end, part);
    k_grad_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(ntiles, part, grad);
  } else {
    cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, st);
  }
  return cudaGetLastError();
}

size_t train_part_floats(int max_pairs) { return (size_t)((max_pairs + TP - 1) / TP) * NPARAM; }

// Adam (Kingma & Ba 2015) on the FP32 master weights; refreshes the bf16 copies
__global__ void k_adam(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float c1, float c2, float beta1, float beta2,
                       float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t adam(float* th, float* m, float* v, const float* g, int t, double lr, float* thq, void* packed,
                 void* packed_tc, cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = float(1.0 - pow(b1, t)), c2 = float(1.0 - pow(b2, t));
  k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(th, m, v, g, float(lr), c1, c2, float(b1), float(b2), 1e-8f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = pack_weights(th, thq, packed, st);   // every inference copy follows the new weights
  if (e != cudaSuccess) return e;
  return pack_weights_tc(th, packed_tc, st);
}

// ---------------------------------------------------------------------------------
// neighbour-list driver
// ---------------------------------------------------------------------------------

cudaError_t bbox(int N, const double* R, double* part_dev, double* out_host, cudaStream_t st) {
  const int blocks = N < 256 * 64 ? (N + 255) / 256 : 64;
  k_bbox<<<blocks, 256, 0, st>>>(N, R, part_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double tmp[64 * 6];
  e = cudaMemcpyAsync(tmp, part_dev, sizeof(double) * 6 * blocks, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int d = 0; d < 3; ++d) {
    out_host[d] = 1e300;
    out_host[3 + d] = -1e300;
  }
  for (int b = 0; b < blocks; ++b)
    for (int d = 0; d < 3; ++d) {
      out_host[d] = fmin(out_host[d], tmp[6 * b + d]);
      out_host[3 + d] = fmax(out_host[3 + d], tmp[6 * b + 3 + d]);
    }
  return cudaSuccess;
}

cudaError_t nb_count_sys(int N, const double* R, const int* sys_of, const int* sys_off, double rc2, int* cnt,
                         cudaStream_t st) {
  k_nb_sys<<<(N + 127) / 128, 128, 0, st>>>(N, R, sys_of, sys_off, rc2, nullptr, cnt, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t nb_fill_sys(int N, const double* R, const int* sys_of, const int* sys_off, double rc2, const int* start,
                        int* tg, int* sr, cudaStream_t st) {
  k_nb_sys<<<(N + 127) / 128, 128, 0, st>>>(N, R, sys_of, sys_off, rc2, start, nullptr, tg, sr);
  return cudaGetLastError();
}

cudaError_t cells_build(int N, const double* R, const double* box, double side, int* dims, int* cell_of,
                        int* cell_cnt, int* cell_start, int* cell_fill, int* items, int* scratch, cudaStream_t st) {
  CellGrid g;
  for (int d = 0; d < 3; ++d) {
    g.lo[d] = box[d];
    g.dim[d] = dims[d];
  }
  g.inv = 1.0 / side;
  const int nc = dims[0] * dims[1] * dims[2];
  cudaError_t e = cudaMemsetAsync(cell_cnt, 0, sizeof(int) * nc, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cell_fill, 0, sizeof(int) * nc, st);
  if (e != cudaSuccess) return e;
  k_cell_count<<<(N + 255) / 256, 256, 0, st>>>(N, R, g, cell_of, cell_cnt);
  e = exclusive_scan(cell_cnt, cell_start, nc, scratch, st);
  if (e != cudaSuccess) return e;
  k_cell_fill<<<(N + 255) / 256, 256, 0, st>>>(N, cell_of, cell_start, cell_fill, items);
  return cudaGetLastError();
}

cudaError_t nb_cells(int N, const double* R, const double* box, double side, const int* dims, const int* cell_of,
                     const int* cell_start, const int* cell_cnt, const int* items, double rc2, const int* start,
                     int* cnt, int* tg, int* sr, int* overflow, cudaStream_t st) {
  CellGrid g;
  for (int d = 0; d < 3; ++d) {
    g.lo[d] = box[d];
    g.dim[d] = dims[d];
  }
  g.inv = 1.0 / side;
  k_nb_cells<<<(N + 127) / 128, 128, 0, st>>>(N, R, g, cell_of, cell_start, cell_cnt, items, rc2, start, cnt, tg,
                                               sr, overflow);
  return cudaGetLastError();
}

cudaError_t features(int P, const double* R, const double* p, const int* tg, const int* sr, double a, float* F,
                     float* FR, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  k_features<<<(P + 127) / 128, 128, 0, st>>>(P, R, p, tg, sr, a, F, FR);
  return cudaGetLastError();
}

}  // namespace mlpk
}  // namespace gbi

namespace gbi {
namespace mlpk {

// dst = sum of parts[0..n) in index order (one thread: n is a few thousand at most)
__global__ void k_sum_into(const double* __restrict__ parts, int n, double* __restrict__ dst) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += parts[i];
  *dst = s;
}

cudaError_t sum_into(const double* parts, int n, double* dst, cudaStream_t st) {
  k_sum_into<<<1, 32, 0, st>>>(parts, n, dst);
  return cudaGetLastError();
}

}  // namespace mlpk
}  // namespace gbi

namespace gbi {
namespace mlpk {

// labels[n][c] = sigma / s0 * (exact - superposition) of (V, Omega); block partial sums
// of the squared differences (for choosing sigma)
__global__ void k_labels(int N, double s0, double sigma, const double* __restrict__ Vx, const double* __restrict__ Ox,
                         const double* __restrict__ Vs, const double* __restrict__ Os, double* __restrict__ labels,
                         double* __restrict__ sq_part) {
  __shared__ double s[256];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double q = 0.0;
  if (n < N) {
    for (int i = 0; i < 3; ++i) {
      const double dv = (Vx[3 * (size_t)n + i] - Vs[3 * (size_t)n + i]) / s0;
      const double dw = (Ox[3 * (size_t)n + i] - Os[3 * (size_t)n + i]) / s0;
      q += dv * dv + dw * dw;
      if (labels != nullptr) {
        labels[(size_t)n * 6 + i] = sigma * dv;
        labels[(size_t)n * 6 + 3 + i] = sigma * dw;
      }
    }
  }
  s[threadIdx.x] = q;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && sq_part != nullptr) sq_part[blockIdx.x] = s[0];
}

cudaError_t labels(int N, double s0, double sigma, const double* Vx, const double* Ox, const double* Vs,
                   const double* Os, double* out, double* sq_part, cudaStream_t st) {
  k_labels<<<(N + 255) / 256, 256, 0, st>>>(N, s0, sigma, Vx, Ox, Vs, Os, out, sq_part);
  return cudaGetLastError();
}

// strain-mode head: labels[n] = sigma / s0 (Q^(2s) of the solve - the one-body Q^(2s)), 0
__global__ void k_labels_q(int N, int h, double s0, double sigma, const double* __restrict__ QHx,
                           const double* __restrict__ QH1, double* __restrict__ labels, double* __restrict__ sq_part) {
  __shared__ double s[256];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double q = 0.0;
  if (n < N) {
    for (int c = 0; c < 5; ++c) {
      const double d = (QHx[(size_t)h * n + c] - QH1[(size_t)h * n + c]) / s0;
      q += d * d;
      if (labels != nullptr) labels[(size_t)n * 6 + c] = sigma * d;
    }
    if (labels != nullptr) labels[(size_t)n * 6 + 5] = 0.0;
  }
  s[threadIdx.x] = q;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && sq_part != nullptr) sq_part[blockIdx.x] = s[0];
}

cudaError_t labels_q(int N, int h, double s0, double sigma, const double* QHx, const double* QH1, double* out,
                     double* sq_part, cudaStream_t st) {
  k_labels_q<<<(N + 255) / 256, 256, 0, st>>>(N, h, s0, sigma, QHx, QH1, out, sq_part);
  return cudaGetLastError();
}

}  // namespace mlpk
}  // namespace gbi
