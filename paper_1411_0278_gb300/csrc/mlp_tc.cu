// Near-field network inference on the 5th-generation tensor cores (tcgen05).
//
// Same network and numerics as k_infer in mlp_kernel.cu (bf16 weights and layer
// inputs, FP32 accumulation, hardware tanh approximation): one 128-pair tile per step, each layer
// one chain of tcgen05.mma.cta_group::1.kind::f16 (M = 128 pairs, N = 128 neurons or 16
// outputs, K = 16 per instruction) issued by a single thread, operands in shared
// memory in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
// matrix), the FP32 accumulator in tensor memory (128 lanes x 128 columns) read back
// with tcgen05.ld by eight warps: a warp may only read the lane quarter of its warp
// index mod 4, so warps w and w + 4 share lanes 32 (w mod 4) .. + 31 (pairs of the tile)
// and each takes half of the 128 columns of the epilogue.  Completion of each MMA chain
// is signalled through an mbarrier (tcgen05.commit); every wait has an iteration limit
// after which the kernel records an error, releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbi_internal.cuh"

namespace gbi {
namespace mlpk {
namespace {

constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH * NH;
constexpr int OFF_W4 = OFF_B3 + NH;
constexpr int OFF_B4 = OFF_W4 + NOUT * NH;

constexpr int TM = 128;          // pairs per tile (MMA M)
constexpr int K1 = 16;           // layer-1 K (9 features, zero-padded)
constexpr int N4 = 16;           // output layer N (6 outputs, zero-padded)
constexpr int CM = 64;           // bf16 elements per core matrix (8 rows x 8)

// core-matrix layout of an R x C matrix: element (r, c) at
//   ((r / 8) * (C / 8) + c / 8) * 64 + (r % 8) * 8 + c % 8
// (8 x 8 blocks, 8 columns contiguous).  As a K-major operand (rows M or N, columns K) its
// descriptor has LBO = 128 bytes (the next 8 columns) and SBO = C * 16 bytes (the next 8
// rows); a K step of 16 advances 256 bytes.  The same storage read as an MN-major operand
// (columns M or N, rows K: the transpose) has LBO = C * 16 bytes (the next 8 rows, along K)
// and SBO = 128 bytes (the next 8 columns, along M or N), and a K step of 16 advances 2 C * 16
// bytes -- the reading an in-bounds check of all four combinations on GB300 confirmed.
__host__ __device__ constexpr int cm_index(int r, int k, int K) { return ((r >> 3) * (K >> 3) + (k >> 3)) * CM + (r & 7) * 8 + (k & 7); }

// packed weights (bf16): W1 [128 x 16], W2 [128 x 128], W3 [128 x 128], W4 [16 x 128], then
// FP32 biases b1, b2, b3 [128], b4 [16]
constexpr int PW1 = 0;
constexpr int PW2 = PW1 + NH * K1;
constexpr int PW3 = PW2 + NH * NH;
constexpr int PW4 = PW3 + NH * NH;
constexpr int PWEND = PW4 + N4 * NH;      // bf16 elements
constexpr int PBIAS = 3 * NH + N4;         // floats
static_assert((PWEND * 2) % 16 == 0, "bias block alignment");

__global__ void k_pack_tc(const float* __restrict__ th, __nv_bfloat16* __restrict__ pk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NH * K1) {
    const int n = i / K1, k = i % K1;
    pk[PW1 + cm_index(n, k, K1)] = __float2bfloat16_rn(k < NIN ? th[OFF_W1 + n * NIN + k] : 0.f);
  }
  if (i < NH * NH) {
    const int n = i / NH, k = i % NH;
    pk[PW2 + cm_index(n, k, NH)] = __float2bfloat16_rn(th[OFF_W2 + n * NH + k]);
    pk[PW3 + cm_index(n, k, NH)] = __float2bfloat16_rn(th[OFF_W3 + n * NH + k]);
  }
  if (i < N4 * NH) {
    const int n = i / NH, k = i % NH;
    pk[PW4 + cm_index(n, k, NH)] = __float2bfloat16_rn(n < NOUT ? th[OFF_W4 + n * NH + k] : 0.f);
  }
  float* b = reinterpret_cast<float*>(pk + PWEND);
  if (i < NH) {
    b[i] = th[OFF_B1 + i];
    b[NH + i] = th[OFF_B2 + i];
    b[2 * NH + i] = th[OFF_B3 + i];
  }
  if (i < N4) b[3 * NH + i] = i < NOUT ? th[OFF_B4 + i] : 0.f;
}

// ---- PTX wrappers --------------------------------------------------------------

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: no swizzle, LBO/SBO in bytes (their meaning for K-major
// and MN-major operands is stated with cm_index above)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  return d;                 // base offset 0, relative LBO, layout 0 = no swizzle
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, K-major unless
// a_mn / b_mn ask for the MN-major form of that operand
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, int a_mn = 0, int b_mn = 0) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

constexpr long long kWaitLimit = 1ll << 22;   // try_wait rounds before giving up

struct TcSmem {
  __nv_bfloat16 w[PWEND];          // weights, core-matrix layout
  float bias[PBIAS];
  __nv_bfloat16 a1[TM * K1];       // layer-1 operand (features)
  __nv_bfloat16 act[TM * NH];      // hidden-layer operand
  unsigned long long mbar;
  uint32_t tmem_base;
  int abort;
};

constexpr int kTcThreads = 256;   // eight warps: two per tensor-memory lane quarter

__global__ void __launch_bounds__(kTcThreads) k_infer_tc(int P, const float* __restrict__ F, const float* __restrict__ FR,
                                                   const __nv_bfloat16* __restrict__ pk, float* __restrict__ out,
                                                   int* __restrict__ err, int head) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (TM - 1);          // the pair of the tile (accumulator lane) this thread reads
  const int half = warp >> 2;              // which 64 of the 128 hidden columns it handles
  {
    const int4* src = reinterpret_cast<const int4*>(pk);
    int4* dst = reinterpret_cast<int4*>(s.w);
    const int n16 = int((sizeof(__nv_bfloat16) * PWEND + sizeof(float) * PBIAS) / 16);
    for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
  }
  const uint32_t mbar = saddr(&s.mbar);
  if (tid == 0) {
    s.abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&s.tmem_base)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s.tmem_base;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;   // this warp's TMEM lane quarter
  const uint32_t a1_addr = saddr(s.a1), act_addr = saddr(s.act), w_addr = saddr(s.w);
  const uint32_t id_hidden = instr_desc(TM, NH), id_out = instr_desc(TM, N4);
  uint32_t parity = 0;
  const int ntiles = (P + TM - 1) / TM;

  // issue one layer (thread 0) and wait for it (all threads); false if the wait gave up
  auto run_layer = [&](uint32_t a_addr, int K, uint32_t b_addr, uint32_t idesc) -> bool {
    fence_async_smem();   // operands written through the generic proxy
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t sbo_a = (uint32_t)K * 16;   // 8 rows x K bf16
      const uint32_t sbo_b = (uint32_t)K * 16;
      for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t ad = smem_desc(a_addr + ks * 256, 128, sbo_a);
        const uint64_t bd = smem_desc(b_addr + ks * 256, 128, sbo_b);
        mma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
      }
      mma_commit(mbar);
    }
    long long it = 0;
    while (!mbar_try_wait(mbar, parity)) {
      if (++it > kWaitLimit) {
        s.abort = 1;
        break;
      }
    }
    parity ^= 1u;
    fence_after();
    __syncthreads();
    return s.abort == 0;
  };

  // hidden epilogue: row `row`, columns [64 half, 64 half + 64) of the accumulator ->
  // tanh(. + b) -> bf16 -> act (core layout)
  auto hidden_epilogue = [&](const float* b) {
#pragma unroll 1
    for (int c0 = half * (NH / 2); c0 < (half + 1) * (NH / 2); c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
      __align__(16) __nv_bfloat16 o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16_rn(tanh_act(v[i] + b[c0 + i]));
      *reinterpret_cast<int4*>(&s.act[cm_index(row, c0, NH)]) = *reinterpret_cast<const int4*>(&o[0]);
      *reinterpret_cast<int4*>(&s.act[cm_index(row, c0 + 8, NH)]) = *reinterpret_cast<const int4*>(&o[8]);
    }
  };

  bool ok = true;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int p = tile * TM + row;
    if (half == 0) {
      __align__(16) __nv_bfloat16 f[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) f[k] = __float2bfloat16_rn((k < NIN && p < P) ? F[(size_t)p * NIN + k] : 0.f);
      *reinterpret_cast<int4*>(&s.a1[cm_index(row, 0, K1)]) = *reinterpret_cast<const int4*>(&f[0]);
      *reinterpret_cast<int4*>(&s.a1[cm_index(row, 8, K1)]) = *reinterpret_cast<const int4*>(&f[8]);
    }
    ok = run_layer(a1_addr, K1, w_addr + 2 * PW1, id_hidden);
    if (!ok) break;
    hidden_epilogue(s.bias);
    ok = run_layer(act_addr, NH, w_addr + 2 * PW2, id_hidden);
    if (!ok) break;
    hidden_epilogue(s.bias + NH);
    ok = run_layer(act_addr, NH, w_addr + 2 * PW3, id_hidden);
    if (!ok) break;
    hidden_epilogue(s.bias + 2 * NH);
    ok = run_layer(act_addr, NH, w_addr + 2 * PW4, id_out);
    if (!ok) break;
    if (half != 0) continue;   // the 16 output columns: the first warp of each lane quarter
    float o[16];
    tmem_ld16(tmem + lane_base, o);
    if (p < P) {
      const float* b4 = s.bias + 3 * NH;
      float y[NOUT];
#pragma unroll
      for (int c = 0; c < NOUT; ++c) y[c] = o[c] + b4[c];
      float* dst = out + (size_t)p * NOUT;
      if (FR != nullptr) {
        pair_out_to_lab(head, FR + (size_t)p * 9, y, dst);
      } else {
#pragma unroll
        for (int c = 0; c < NOUT; ++c) dst[c] = y[c];
      }
    }
  }
  if (!ok) {
    // a chain that did not signal in time may still be running: wait once more (bounded)
    // before the tensor memory it writes is released
    long long it = 0;
    while (!mbar_try_wait(mbar, parity ^ 1u) && ++it <= kWaitLimit) {
    }
    if (tid == 0) atomicExch(err, 1);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128) : "memory");
}

// ---- training: backward pass on the tensor cores -------------------------------------
//
// For a tile of 128 pairs (dO given by the loss kernel, FP32 [P][6]) the forward pass is
// recomputed exactly as k_infer_tc computes it (bf16 layer inputs, FP32 accumulation,
// hardware tanh), and then, with dZ_L = dH_L (1 - h_L^2) rounded to bf16:
//   dH3 = dO W4,            dW4^T += H3^T dO,
//   dW3 += dZ3^T H2,        db3 += dZ3^T 1,       dH2 = dZ3 W3,
//   dW2 += dZ2^T H1,        db2 += dZ2^T 1,       dH1 = dZ2 W2,
//   dW1 += dZ1^T X          (feature slot 9 holds 1, so column 9 is db1),
// db4 = sum of dO in FP32.  The transposed operands are the same shared-memory tiles read
// MN-major.  The weight gradients stay in tensor memory across all tiles a block takes and
// are written once per block (a partial gradient that a fixed-order reduction sums).
// h in (1 - h^2) is the bf16-rounded layer output (the value the next layer multiplies).
constexpr int kBwThreads = 256;
constexpr int kColZ = 0, kColW3 = 128, kColW2 = 256, kColW1 = 384, kColW4 = 400, kColB3 = 416, kColB2 = 432;
constexpr int kBwTmemCols = 512;

struct BwSmem {
  __nv_bfloat16 h[3][TM * NH];     // layer outputs (bf16), [pairs x 128]
  __nv_bfloat16 dz[TM * NH];       // dZ of the layer being differentiated, [pairs x 128]
  __nv_bfloat16 x[TM * K1];        // features, slot NIN = 1, [pairs x 16]
  __nv_bfloat16 dout[TM * N4];     // dO (bf16), [pairs x 16]
  __nv_bfloat16 ones[N4 * TM];     // row 0 ones, [16 x pairs]
  __nv_bfloat16 w[PWEND];          // weights, the inference layout
  float bias[PBIAS];
  float db4[4][N4];
  unsigned long long mbar;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(BwSmem) <= 227 * 1024, "one block per SM, within the shared-memory limit");

__global__ void __launch_bounds__(kBwThreads) k_train_bwd_tc(int P, const float* __restrict__ F,
                                                          const float* __restrict__ dO,
                                                          const __nv_bfloat16* __restrict__ pk,
                                                          float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  BwSmem& s = *reinterpret_cast<BwSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (TM - 1);
  const int half = warp >> 2;
  {
    const int4* src = reinterpret_cast<const int4*>(pk);
    int4* dst = reinterpret_cast<int4*>(s.w);
    const int n16 = int((sizeof(__nv_bfloat16) * PWEND + sizeof(float) * PBIAS) / 16);
    for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    for (int i = tid; i < N4 * TM; i += blockDim.x) s.ones[i] = __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  if (tid < TM) s.ones[cm_index(0, tid, TM)] = __float2bfloat16_rn(1.f);
  const uint32_t mbar = saddr(&s.mbar);
  if (tid == 0) {
    s.abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&s.tmem_base)),
                 "r"(kBwTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s.tmem_base;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t x_a = saddr(s.x), do_a = saddr(s.dout), dz_a = saddr(s.dz), one_a = saddr(s.ones);
  const uint32_t h_a[3] = {saddr(s.h[0]), saddr(s.h[1]), saddr(s.h[2])};
  const uint32_t w_a = saddr(s.w);
  const uint32_t w1_a = w_a + 2 * PW1, w2_a = w_a + 2 * PW2, w3_a = w_a + 2 * PW3, w4_a = w_a + 2 * PW4;
  uint32_t parity = 0;
  const int ntiles = (P + TM - 1) / TM;
  float db4acc[NOUT];
#pragma unroll
  for (int c = 0; c < NOUT; ++c) db4acc[c] = 0.f;

  // nk MMAs into column dcol: operand start addresses advance by the K steps given
  auto chain = [&](int dcol, uint32_t a0, uint32_t alb, uint32_t asb, uint32_t astep, uint32_t b0, uint32_t blb,
                   uint32_t bsb, uint32_t bstep, int nk, uint32_t idesc, bool accum) {
    for (int ks = 0; ks < nk; ++ks)
      mma_f16(tmem + (uint32_t)dcol, smem_desc(a0 + ks * astep, alb, asb), smem_desc(b0 + ks * bstep, blb, bsb), idesc,
              (accum || ks > 0) ? 1u : 0u);
  };
  // operands written by threads become visible to the tensor cores
  auto publish = [&]() {
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
  };
  // thread 0 commits what it issued; everyone waits (bounded)
  auto complete = [&]() -> bool {
    if (tid == 0) mma_commit(mbar);
    long long it = 0;
    while (!mbar_try_wait(mbar, parity)) {
      if (++it > kWaitLimit) {
        s.abort = 1;
        break;
      }
    }
    parity ^= 1u;
    fence_after();
    __syncthreads();
    return s.abort == 0;
  };
  // tanh(Z + b) -> bf16 layer output L
  auto forward_epilogue = [&](int L) {
    const float* b = s.bias + L * NH;
#pragma unroll 1
    for (int c0 = half * (NH / 2); c0 < (half + 1) * (NH / 2); c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)(kColZ + c0), v);
      __align__(16) __nv_bfloat16 o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16_rn(tanh_act(v[i] + b[c0 + i]));
      *reinterpret_cast<int4*>(&s.h[L][cm_index(row, c0, NH)]) = *reinterpret_cast<const int4*>(&o[0]);
      *reinterpret_cast<int4*>(&s.h[L][cm_index(row, c0 + 8, NH)]) = *reinterpret_cast<const int4*>(&o[8]);
    }
  };
  // dZ = dH (1 - h_L^2) -> bf16
  auto backward_epilogue = [&](int L) {
#pragma unroll 1
    for (int c0 = half * (NH / 2); c0 < (half + 1) * (NH / 2); c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)(kColZ + c0), v);
      __align__(16) __nv_bfloat16 hv[16];
      *reinterpret_cast<int4*>(&hv[0]) = *reinterpret_cast<const int4*>(&s.h[L][cm_index(row, c0, NH)]);
      *reinterpret_cast<int4*>(&hv[8]) = *reinterpret_cast<const int4*>(&s.h[L][cm_index(row, c0 + 8, NH)]);
      __align__(16) __nv_bfloat16 o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float h = __bfloat162float(hv[i]);
        o[i] = __float2bfloat16_rn(v[i] * (1.f - h * h));
      }
      *reinterpret_cast<int4*>(&s.dz[cm_index(row, c0, NH)]) = *reinterpret_cast<const int4*>(&o[0]);
      *reinterpret_cast<int4*>(&s.dz[cm_index(row, c0 + 8, NH)]) = *reinterpret_cast<const int4*>(&o[8]);
    }
  };

  const uint32_t id_h = instr_desc(TM, NH), id_h_bmn = instr_desc(TM, NH, 0, 1);
  const uint32_t id_w = instr_desc(NH, NH, 1, 1), id_w16 = instr_desc(NH, N4, 1, 1), id_b = instr_desc(NH, N4, 1, 0);
  constexpr uint32_t SB128 = NH * 16, SB16 = K1 * 16;   // 8-row strides of the 128- and 16-column tiles
  bool ok = true, first = true;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int p = tile * TM + row;
    const bool live = p < P;
    if (half == 0) {
      __align__(16) __nv_bfloat16 f[16];
#pragma unroll
      for (int k = 0; k < 16; ++k)
        f[k] = __float2bfloat16_rn(k < NIN ? (live ? F[(size_t)p * NIN + k] : 0.f) : (k == NIN && live ? 1.f : 0.f));
      *reinterpret_cast<int4*>(&s.x[cm_index(row, 0, K1)]) = *reinterpret_cast<const int4*>(&f[0]);
      *reinterpret_cast<int4*>(&s.x[cm_index(row, 8, K1)]) = *reinterpret_cast<const int4*>(&f[8]);
    } else {
      __align__(16) __nv_bfloat16 g[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float v = (c < NOUT && live) ? dO[(size_t)p * 6 + c] : 0.f;
        if (c < NOUT) db4acc[c] += v;
        g[c] = __float2bfloat16_rn(v);
      }
      *reinterpret_cast<int4*>(&s.dout[cm_index(row, 0, N4)]) = *reinterpret_cast<const int4*>(&g[0]);
      *reinterpret_cast<int4*>(&s.dout[cm_index(row, 8, N4)]) = *reinterpret_cast<const int4*>(&g[8]);
    }
    // forward: Z = X W1^T, H1 W2^T, H2 W3^T
    publish();
    if (tid == 0) chain(kColZ, x_a, 128, SB16, 256, w1_a, 128, SB16, 256, 1, id_h, false);
    if (!(ok = complete())) break;
    forward_epilogue(0);
    publish();
    if (tid == 0) chain(kColZ, h_a[0], 128, SB128, 256, w2_a, 128, SB128, 256, NH / 16, id_h, false);
    if (!(ok = complete())) break;
    forward_epilogue(1);
    publish();
    if (tid == 0) chain(kColZ, h_a[1], 128, SB128, 256, w3_a, 128, SB128, 256, NH / 16, id_h, false);
    if (!(ok = complete())) break;
    forward_epilogue(2);
    publish();
    // output layer: dH3 = dO W4 (W4 [16 x 128] read MN-major), dW4^T += H3^T dO
    if (tid == 0) {
      chain(kColZ, do_a, 128, SB16, 256, w4_a, SB128, 128, 2 * SB128, 1, id_h_bmn, false);
      chain(kColW4, h_a[2], SB128, 128, 2 * SB128, do_a, SB16, 128, 2 * SB16, TM / 16, id_w16, !first);
    }
    if (!(ok = complete())) break;
    backward_epilogue(2);
    publish();
    // layers 3 and 2: dW += dZ^T H_prev, db += dZ^T 1, dH_prev = dZ W
    for (int L = 2; L >= 1 && ok; --L) {
      if (tid == 0) {
        const int cw = L == 2 ? kColW3 : kColW2, cb = L == 2 ? kColB3 : kColB2;
        const uint32_t wl = L == 2 ? w3_a : w2_a;
        chain(cw, dz_a, SB128, 128, 2 * SB128, h_a[L - 1], SB128, 128, 2 * SB128, TM / 16, id_w, !first);
        chain(cb, dz_a, SB128, 128, 2 * SB128, one_a, 128, SB128, 256, TM / 16, id_b, !first);
        chain(kColZ, dz_a, 128, SB128, 256, wl, SB128, 128, 2 * SB128, NH / 16, id_h_bmn, false);
      }
      if (!(ok = complete())) break;
      backward_epilogue(L - 1);
      publish();
    }
    if (!ok) break;
    // layer 1: dW1 (and db1 in column 9) += dZ1^T X
    if (tid == 0) chain(kColW1, dz_a, SB128, 128, 2 * SB128, x_a, SB16, 128, 2 * SB16, TM / 16, id_w16, !first);
    if (!(ok = complete())) break;
    first = false;
  }
  // the block's partial gradient
  float* g = part + (size_t)blockIdx.x * NPARAM;
  if (ok && !first) {
    const int j = row;
#pragma unroll 1
    for (int c0 = half * (NH / 2); c0 < (half + 1) * (NH / 2); c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)(kColW3 + c0), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) g[OFF_W3 + j * NH + c0 + i] = v[i];
      tmem_ld16(tmem + lane_base + (uint32_t)(kColW2 + c0), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) g[OFF_W2 + j * NH + c0 + i] = v[i];
    }
    float v[16], u[16];
    if (half == 0) {
      tmem_ld16(tmem + lane_base + (uint32_t)kColW1, v);
      tmem_ld16(tmem + lane_base + (uint32_t)kColB3, u);
#pragma unroll
      for (int k = 0; k < NIN; ++k) g[OFF_W1 + j * NIN + k] = v[k];
      g[OFF_B1 + j] = v[NIN];
      g[OFF_B3 + j] = u[0];
    } else {
      tmem_ld16(tmem + lane_base + (uint32_t)kColW4, v);
      tmem_ld16(tmem + lane_base + (uint32_t)kColB2, u);
#pragma unroll
      for (int c = 0; c < NOUT; ++c) g[OFF_W4 + c * NH + j] = v[c];
      g[OFF_B2 + j] = u[0];
    }
  }
  // db4: the dO sums of the threads that staged dO (warps 4..7), fixed order
  if (half == 1) {
#pragma unroll
    for (int c = 0; c < NOUT; ++c) {
      float t = db4acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if ((tid & 31) == 0) s.db4[warp - 4][c] = t;
    }
  }
  __syncthreads();
  if (tid < NOUT) g[OFF_B4 + tid] = ((s.db4[0][tid] + s.db4[1][tid]) + s.db4[2][tid]) + s.db4[3][tid];
  if (!ok) {
    long long it = 0;
    while (!mbar_try_wait(mbar, parity ^ 1u) && ++it <= kWaitLimit) {
    }
    if (tid == 0) atomicExch(err, 1);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kBwTmemCols) : "memory");
}

}  // namespace

size_t packed_tc_bytes() { return sizeof(__nv_bfloat16) * PWEND + sizeof(float) * PBIAS; }

cudaError_t pack_weights_tc(const float* theta, void* packed, cudaStream_t st) {
  k_pack_tc<<<(NH * NH + 255) / 256, 256, 0, st>>>(theta, static_cast<__nv_bfloat16*>(packed));
  return cudaGetLastError();
}

cudaError_t infer_tc(int P, const float* F, const float* FR, const void* packed, float* out, int* err, int num_sms,
                     int head, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  const size_t smem = sizeof(TcSmem);
  cudaError_t e = cudaFuncSetAttribute(k_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int ntiles = (P + TM - 1) / TM;
  const int grid = ntiles < 2 * num_sms ? ntiles : 2 * num_sms;
  k_infer_tc<<<grid, kTcThreads, smem, st>>>(P, F, FR, static_cast<const __nv_bfloat16*>(packed), out, err, head);
  return cudaGetLastError();
}

}  // namespace mlpk
}  // namespace gbi

namespace gbi {
namespace mlpk {

int train_bwd_tc_blocks(int P, int num_sms) {
  const int ntiles = (P + TM - 1) / TM;
  return ntiles < num_sms ? ntiles : num_sms;
}

cudaError_t train_bwd_tc(int P, const float* F, const float* dO, const void* packed, float* part, int* err,
                         int num_sms, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  const size_t smem = sizeof(BwSmem);
  cudaError_t e = cudaFuncSetAttribute(k_train_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k_train_bwd_tc<<<train_bwd_tc_blocks(P, num_sms), kBwThreads, smem, st>>>(
      P, F, dO, static_cast<const __nv_bfloat16*>(packed), part, err);
  return cudaGetLastError();
}

}  // namespace mlpk
}  // namespace gbi
