// Learned warm start: the multilayer perceptron of the nrto_mlp_* entry points (include/nrto.h).
//
// The paper names learning a warm start for the inner solver as future work and fixes no network;
// this file implements a GELU MLP trained by masked mean-squared error with Adam.  Weights are
// kept as FP32 master copies (optimizer) and as bf16 copies for the tensor cores; activations
// between layers are bf16, pre-activations FP32.  Every matrix product (forward, input gradients,
// weight gradients) is one tcgen05 GEMM kernel with bf16 operands and an FP32 accumulator in
// tensor memory, D = A·Bᵀ with both operands K-major (contraction dimension contiguous):
//   forward     Z_{l+1} = H_l · W_lᵀ          A = H_l [B][d_l],        B = W_l [d_{l+1}][d_l]
//   input grad  dH_l    = dZ_{l+1} · W_l      A = dZ_{l+1} [B][d_{l+1}], B = W_lᵀ [d_l][d_{l+1}]
//   weight grad dW_l    = dZ_{l+1}ᵀ · H_l     A = dZ_{l+1}ᵀ [d_{l+1}][B], B = H_lᵀ [d_l][B]
// (transposed activations are produced by a tiled transpose kernel).  Bias, GELU and GELU'
// are fused into the GEMM epilogue.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/nrto.h"
#include "umma.cuh"

void nrto_internal_set_error(const std::string& msg);   // api.cu

using namespace nrto;
typedef __nv_bfloat16 bf16;

namespace {

struct MlpError {
  nrto_status st;
  std::string msg;
};

#define MK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) throw MlpError{NRTO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

void mfail(nrto_status s, const std::string& m) { throw MlpError{s, m}; }

// ---------------------------------------------------------------------------------------------
// GEMM: D[M][N] = A[M][K] · B[N][K]ᵀ, bf16 operands, FP32 accumulator in TMEM.
// CTA tile 128 × BN, 64-wide K stages (one 128-byte swizzle row), GEMM_STAGES-deep TMA pipeline.
// Thread 0 issues the bulk tensor loads, thread 32 issues the MMAs (one per K = 16), all four
// warps run the epilogue from TMEM (warp w owns accumulator rows 32w .. 32w+31).
// ---------------------------------------------------------------------------------------------
constexpr int GEMM_STAGES = 4;
// column splits of the persistent output-layer GEMM's epilogue (4·NRTO_GEMM_CS epilogue warps)
#ifndef NRTO_GEMM_CS
#define NRTO_GEMM_CS 4
#endif
enum : int { EPI_BIAS_GELU = 0, EPI_BIAS = 1, EPI_GELU_BWD = 2, EPI_F32 = 3 };

struct EpiArgs {
  int M, N;
  const float* bias;     // [N]                      (EPI_BIAS_GELU, EPI_BIAS)
  float* out_f32;        // Z / Y / dW rows, ld_f32  (EPI_BIAS_GELU, EPI_BIAS, EPI_F32)
  int ld_f32;
  bf16* out_bf16;        // H / dZ rows, ld_bf16     (EPI_BIAS_GELU, EPI_GELU_BWD)
  int ld_bf16;
  const float* zin;      // Z rows for GELU', ld_zin (EPI_GELU_BWD)
  int ld_zin;
  int* err;              // set to 1 when a pipeline wait gave up
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// STG pipeline stages; with two stages a CTA needs half the shared memory, so two CTAs share an SM
// and one's epilogue overlaps the other's loads and MMAs (the short-K output layer).
template <int BN, int STG = GEMM_STAGES>
constexpr size_t gemm_smem_bytes() { return 1024 + (size_t)STG * (128 * 128 + BN * 128); }

template <int BN, int EPI, int STG = GEMM_STAGES>
__global__ void __launch_bounds__(128, STG == 2 ? 2 : 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int K, EpiArgs ep) {
  constexpr int GEMM_STAGES = STG;
  extern __shared__ uint8_t smem_raw[];
  constexpr int A_BYTES = 128 * 128, B_BYTES = BN * 128, STAGE = A_BYTES + B_BYTES;
  __shared__ __align__(8) uint64_t full[GEMM_STAGES], empty[GEMM_STAGES], accb;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
  const int nk = (K + 63) / 64;
  if (warp == 0) {
    tmem_alloc(&tmem_base, BN);
    tmem_relinquish();
  }
  if (tid == 32) {
    for (int s = 0; s < GEMM_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(&accb, 1);
    fence_mbar_init();
    s_err = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  int issued = 0;   // stages the producer has issued loads for (thread 0)
  if (tid == 0) {
    // producer: bulk tensor loads of the A and B stages
    for (int k = 0; k < nk; ++k) {
      const int s = k % GEMM_STAGES;
      if (k >= GEMM_STAGES && !mbar_wait_bounded(&empty[s], (uint32_t)((k / GEMM_STAGES) - 1) & 1u)) {
        s_err = 1;
        break;
      }
      uint8_t* sa = base + (size_t)s * STAGE;
      mbar_arrive_expect_tx(&full[s], STAGE);
      tma_load_2d(sa, &ta, k * 64, m0, &full[s]);
      tma_load_2d(sa + A_BYTES, &tb, k * 64, n0, &full[s]);
      issued = k + 1;
    }
  } else if (tid == 32) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(128, BN);
    for (int k = 0; k < nk; ++k) {
      const int s = k % GEMM_STAGES;
      if (!mbar_wait_bounded(&full[s], (uint32_t)(k / GEMM_STAGES) & 1u)) {
        s_err = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(base + (size_t)s * STAGE), sb = sa + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma_bf16(tmem, sdesc_k_sw128(sa + kk * 32), sdesc_k_sw128(sb + kk * 32), idesc, (k | kk) != 0 ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(&accb);
  }
  if (!mbar_wait_bounded(&accb, 0)) s_err = 1;
  __syncwarp();
  tc_fence_after();

  // epilogue: TMEM → registers → global
  const int row = m0 + warp * 32 + lane;
  if constexpr (EPI == EPI_BIAS || EPI == EPI_F32) {
    // FP32 outputs: each warp turns its 32 × 32 slices around in shared memory (the stage buffers are
    // idle once the accumulator is complete) so that a store instruction writes 32 consecutive
    // columns of one row, with the bias added per column
    float* tbuf = reinterpret_cast<float*>(base) + warp * (32 * 33);
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      float v[32];
      tmem_ld_32x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
      const int nb = n0 + c * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) tbuf[lane * 33 + j] = v[j];
      __syncwarp();
      const int n = nb + lane;
      float bv = 0.0f;
      if constexpr (EPI == EPI_BIAS) bv = n < ep.N ? ep.bias[n] : 0.0f;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int rr = m0 + warp * 32 + r;
        if (rr < ep.M && n < ep.N) ep.out_f32[(long long)rr * ep.ld_f32 + n] = tbuf[r * 33 + lane] + bv;
      }
      __syncwarp();
    }
  }
#pragma unroll 1
  for (int c = 0; c < ((EPI == EPI_BIAS || EPI == EPI_F32) ? 0 : BN / 32); ++c) {
    float v[32];
    tmem_ld_32x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
    const int nb = n0 + c * 32;
    // full 32-column chunks with 16-byte aligned rows: vector stores; ragged edges: scalar
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    bool vec = (nb + 32 <= ep.N);
    if constexpr (EPI == EPI_BIAS_GELU)
      vec = vec && (ep.ld_f32 % 4 == 0) && (ep.ld_bf16 % 8 == 0) && al16(ep.out_f32) && al16(ep.out_bf16);
    else if constexpr (EPI == EPI_GELU_BWD)
      vec = vec && (ep.ld_bf16 % 8 == 0) && (ep.ld_zin % 4 == 0) && al16(ep.out_bf16) && al16(ep.zin);
    else vec = vec && (ep.ld_f32 % 4 == 0) && al16(ep.out_f32);
    if (row < ep.M && vec) {
      if constexpr (EPI == EPI_BIAS_GELU) {
        float4* zo = reinterpret_cast<float4*>(ep.out_f32 + (long long)row * ep.ld_f32 + nb);
        uint4* ho = reinterpret_cast<uint4*>(ep.out_bf16 + (long long)row * ep.ld_bf16 + nb);
#pragma unroll
        for (int j8 = 0; j8 < 4; ++j8) {
          float z[8];
          __align__(16) bf16 h[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            z[t] = v[j8 * 8 + t] + ep.bias[nb + j8 * 8 + t];
            h[t] = __float2bfloat16_rn(gelu_f(z[t]));
          }
          zo[2 * j8] = make_float4(z[0], z[1], z[2], z[3]);
          zo[2 * j8 + 1] = make_float4(z[4], z[5], z[6], z[7]);
          ho[j8] = *reinterpret_cast<const uint4*>(h);
        }
      } else if constexpr (EPI == EPI_GELU_BWD) {
        const float4* zi = reinterpret_cast<const float4*>(ep.zin + (long long)row * ep.ld_zin + nb);
        uint4* ho = reinterpret_cast<uint4*>(ep.out_bf16 + (long long)row * ep.ld_bf16 + nb);
#pragma unroll
        for (int j8 = 0; j8 < 4; ++j8) {
          const float4 za = zi[2 * j8], zb = zi[2 * j8 + 1];
          const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
          __align__(16) bf16 h[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) h[t] = __float2bfloat16_rn(v[j8 * 8 + t] * gelu_grad_f(zz[t]));
          ho[j8] = *reinterpret_cast<const uint4*>(h);
        }
      } else {
        float4* o = reinterpret_cast<float4*>(ep.out_f32 + (long long)row * ep.ld_f32 + nb);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          float a[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            a[t] = v[j4 * 4 + t];
            if constexpr (EPI == EPI_BIAS) a[t] += ep.bias[nb + j4 * 4 + t];
          }
          o[j4] = make_float4(a[0], a[1], a[2], a[3]);
        }
      }
    } else if (row < ep.M && nb < ep.N) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = nb + j;
        if (n < ep.N) {
          float a = v[j];
          if constexpr (EPI == EPI_BIAS_GELU) {
            a += ep.bias[n];
            ep.out_f32[(long long)row * ep.ld_f32 + n] = a;
            ep.out_bf16[(long long)row * ep.ld_bf16 + n] = __float2bfloat16_rn(gelu_f(a));
          } else if constexpr (EPI == EPI_BIAS) {
            ep.out_f32[(long long)row * ep.ld_f32 + n] = a + ep.bias[n];
          } else if constexpr (EPI == EPI_GELU_BWD) {
            ep.out_bf16[(long long)row * ep.ld_bf16 + n] =
                __float2bfloat16_rn(a * gelu_grad_f(ep.zin[(long long)row * ep.ld_zin + n]));
          } else {
            ep.out_f32[(long long)row * ep.ld_f32 + n] = a;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // After a wait gave up (any thread), tensor loads the producer issued may still be landing in this
  // CTA's shared memory: wait (bounded) for the last stages it issued before the CTA exits.
  if (tid == 0 && s_err) {
    for (int k = issued > GEMM_STAGES ? issued - GEMM_STAGES : 0; k < issued; ++k)
      (void)mbar_wait_bounded(&full[k % GEMM_STAGES], (uint32_t)(k / GEMM_STAGES) & 1u);
  }
  __syncwarp();
  if (warp == 0) tmem_dealloc(tmem, BN);
  if (tid == 0 && s_err) atomicExch(ep.err, 1);
}

// ---------------------------------------------------------------------------------------------
// Persistent GEMM for FP32 outputs with a bias (the output layer, wide N and short K): one CTA per
// SM walks the 128 × BN tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (m-blocks fastest, so the
// CTAs working at a time share the B tile in L2).  Warp 4·CS (lane 0) issues the bulk tensor loads
// through an STG-deep stage ring that runs on across tiles; warp 4·CS+1 (lane 0) issues the MMAs into
// one of two TMEM accumulators (columns [0, BN) and [BN, 2 BN)); warps 0 .. 4·CS-1 run the epilogue
// of tile i while the MMAs of tile i+1 run, warp w on TMEM lane quarter w % 4 and column split w / 4
// (several warps per quarter, since the FP32 stores set the epilogue's pace).  Accumulator a is full
// when the MMAs of its tile have completed (acc_full[a], tcgen05.commit) and empty again when every
// epilogue warp has read it (acc_empty[a], 4·CS arrivals).  The epilogue turns each warp's 32 × 32
// slices around in its shared buffer so that a store writes 32 consecutive columns of one row.
// Results equal k_gemm_bf16's (the same MMA order per tile).  Every wait is bounded; after one
// gives up, the CTA waits (bounded) for its issued loads and MMAs before it frees the TMEM.
// ---------------------------------------------------------------------------------------------
// CS column splits of the epilogue: 4·CS epilogue warps, then the producer and the MMA warps.
template <int BN, int STG, int CS>
constexpr size_t gemm_persistent_smem_bytes() { return 1024 + (size_t)STG * (128 * 128 + BN * 128) + 4 * CS * 32 * 33 * 4; }

template <int BN, int STG, int CS>
__global__ void __launch_bounds__(32 * (4 * CS + 2), 1)
k_gemm_bf16_persistent(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int K,
                       int tiles_m, int tiles, EpiArgs ep) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int A_BYTES = 128 * 128, B_BYTES = BN * 128, STAGE = A_BYTES + B_BYTES;
  __shared__ __align__(8) uint64_t full[STG], empty[STG], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_err;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* tbuf_all = reinterpret_cast<float*>(base + (size_t)STG * STAGE);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = (K + 63) / 64;
  constexpr int NEPI = 4 * CS, PROD = 32 * NEPI, MMA = 32 * NEPI + 32;   // lane 0 of the last two warps
  static_assert((BN / 32) % CS == 0, "the column splits must divide the tile's 32-column chunks");
  if (warp == NEPI) {
    tmem_alloc(&tmem_base, 2 * BN);
    tmem_relinquish();
  }
  if (tid == MMA) {
    for (int s = 0; s < STG; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&acc_full[a], 1); mbar_init(&acc_empty[a], NEPI); }
    mbar_init(&mma_done, 1);
    fence_mbar_init();
    s_err = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;   // stages the producer has issued loads for
  if (tid == PROD) {
    int g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int m0 = (t % tiles_m) * 128, n0 = (t / tiles_m) * BN;
      for (int k = 0; k < nk; ++k, ++g) {
        const int s = g % STG;
        if (g >= STG && !mbar_wait_bounded(&empty[s], (uint32_t)((g / STG) - 1) & 1u)) {
          s_err = 1;
          ok = false;
          break;
        }
        uint8_t* sa = base + (size_t)s * STAGE;
        mbar_arrive_expect_tx(&full[s], STAGE);
        tma_load_2d(sa, &ta, k * 64, m0, &full[s]);
        tma_load_2d(sa + A_BYTES, &tb, k * 64, n0, &full[s]);
        issued = g + 1;
      }
    }
  } else if (tid == MMA) {
    constexpr uint32_t idesc = idesc_bf16_f32(128, BN);
    int g = 0, li = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++li) {
      const int a = li & 1;
      if (li >= 2 && !mbar_wait_bounded(&acc_empty[a], (uint32_t)((li >> 1) - 1) & 1u)) {
        s_err = 1;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(a * BN);
      for (int k = 0; k < nk; ++k, ++g) {
        const int s = g % STG;
        if (!mbar_wait_bounded(&full[s], (uint32_t)(g / STG) & 1u)) {
          s_err = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(base + (size_t)s * STAGE), sb = sa + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          umma_bf16(d, sdesc_k_sw128(sa + kk * 32), sdesc_k_sw128(sb + kk * 32), idesc, (k | kk) != 0 ? 1u : 0u);
        umma_commit(&empty[s]);
      }
      if (ok) umma_commit(&acc_full[a]);
    }
    // every MMA this thread issued has completed once mma_done fires
    umma_commit(&mma_done);
    if (!mbar_wait_bounded(&mma_done, 0)) s_err = 1;
  } else if (warp < NEPI) {
    float* tbuf = tbuf_all + warp * (32 * 33);
    const int q = warp & 3, h = warp >> 2;   // TMEM lane quarter, column split
    constexpr int CPW = BN / 32 / CS;        // 32-column chunks per warp
    int li = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++li) {
      const int a = li & 1;
      int got = 1;
      if (lane == 0) got = mbar_wait_bounded(&acc_full[a], (uint32_t)(li >> 1) & 1u) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        if (lane == 0) s_err = 1;
        break;
      }
      tc_fence_after();
      const int m0 = (t % tiles_m) * 128, n0 = (t / tiles_m) * BN;
#pragma unroll 1
      for (int c = h * CPW; c < (h + 1) * CPW; ++c) {
        float v[32];
        tmem_ld_32x32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN + c * 32), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) tbuf[lane * 33 + j] = v[j];
        __syncwarp();
        const int n = n0 + c * 32 + lane;
        const float bv = n < ep.N ? ep.bias[n] : 0.0f;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const int rr = m0 + q * 32 + r;
          if (rr < ep.M && n < ep.N) ep.out_f32[(long long)rr * ep.ld_f32 + n] = tbuf[r * 33 + lane] + bv;
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == PROD && s_err) {
    for (int k = issued > STG ? issued - STG : 0; k < issued; ++k)
      (void)mbar_wait_bounded(&full[k % STG], (uint32_t)(k / STG) & 1u);
  }
  __syncthreads();
  if (warp == NEPI) tmem_dealloc(tmem, 2 * BN);
  if (tid == 0 && s_err) atomicExch(ep.err, 1);
}


// ---------------------------------------------------------------------------------------------
// elementwise / small kernels
// ---------------------------------------------------------------------------------------------
// fp32 [rows][cols] → bf16 [rows][ldo] with zero padding columns cols .. ldo-1
__global__ void k_to_bf16_pad(const float* in, int rows, int cols, bf16* out, int ldo) {
  const long long n = (long long)rows * ldo;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(q / ldo), c = (int)(q % ldo);
    out[q] = __float2bfloat16_rn(c < cols ? in[(long long)r * cols + c] : 0.0f);
  }
}

// bf16 [rows][cols] (leading dim ld_in) → [cols][rows] (leading dim ld_out), 32×32 tiles
__global__ void k_transpose_bf16(const bf16* in, int rows, int cols, int ld_in, bf16* out, int ld_out) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? in[(long long)r * ld_in + c] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[(long long)c * ld_out + r] = tile[threadIdx.x][i];
  }
}

// dY = 2·mask·(Y - T)/n_mask (bf16) and Σ mask·(Y - T)² (double, accumulated)
__global__ void k_mse_grad(const float* Y, const float* Tg, const float* mask, long long n, double inv_n, bf16* dY,
                           double* loss) {
  double acc = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const float d = mask[q] * (Y[q] - Tg[q]);
    acc += (double)d * (double)(Y[q] - Tg[q]);
    dY[q] = __float2bfloat16_rn((float)(2.0 * inv_n) * d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s);
  }
}

// db[n] = Σ_m dZ[m][n]
__global__ void k_colsum_bf16(const bf16* dZ, int rows, int cols, int ld, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  float s = 0.0f;
  for (int m = 0; m < rows; ++m) s += __bfloat162float(dZ[(long long)m * ld + n]);
  db[n] = s;
}

// Adam on the flat FP32 parameters (bias-corrected moments)
__global__ void k_adam(float* theta, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    theta[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

// bf16 copies of one layer's weights W [out][in] (FP32 master): Wt [out][ld_t] (zero padded) and,
// if Wkn != null, its transpose Wkn [in][out].
__global__ void k_weights_bf16(const float* W, int out, int in, bf16* Wt, int ld_t, bf16* Wkn) {
  const long long n = (long long)out * ld_t;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(q / ld_t), i = (int)(q % ld_t);
    const bf16 w = __float2bfloat16_rn(i < in ? W[(long long)o * in + i] : 0.0f);
    Wt[q] = w;
    if (Wkn && i < in) Wkn[(long long)i * out + o] = w;
  }
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    MK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) mfail(NRTO_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return g_encode;
}

// K-major bf16 matrix [rows][k_ext] with leading dimension ld (elements), box 64 × box_rows, 128-byte swizzle.
CUtensorMap make_map(const bf16* ptr, long long rows, long long k_ext, long long ld, int box_rows) {
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || (ld * 2) % 16 != 0) mfail(NRTO_ERR_INVALID, "internal: TMA alignment");
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  cuuint64_t dims[2] = {(cuuint64_t)k_ext, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1u, 1u};
  CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) mfail(NRTO_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

template <int BN, int EPI, int STG = GEMM_STAGES>
void launch_gemm(cudaStream_t st, const bf16* A, long long lda, const bf16* B, long long ldb, int M, int N, int K,
                 const EpiArgs& ep) {
  static_assert(STG >= 2 && (STG > 2 || BN <= 256), "two resident CTAs need BN <= 256 TMEM columns each");
  const CUtensorMap ta = make_map(A, M, K, lda, 128);
  const CUtensorMap tb = make_map(B, N, K, ldb, BN);
  auto kern = k_gemm_bf16<BN, EPI, STG>;
  static bool attr_set = false;   // per template instance
  if (!attr_set) {
    MK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes<BN, STG>()));
    attr_set = true;
  }
  dim3 grid((M + 127) / 128, (N + BN - 1) / BN);
  kern<<<grid, 128, gemm_smem_bytes<BN, STG>(), st>>>(ta, tb, K, ep);
  MK(cudaGetLastError());
}

template <int BN, int STG, int CS>
void launch_gemm_persistent(cudaStream_t st, const bf16* A, long long lda, const bf16* B, long long ldb, int M, int N,
                            int K, const EpiArgs& ep) {
  static_assert(2 * BN <= 512, "two accumulators of BN columns must fit the 512 TMEM columns");
  const CUtensorMap ta = make_map(A, M, K, lda, 128);
  const CUtensorMap tb = make_map(B, N, K, ldb, BN);
  auto kern = k_gemm_bf16_persistent<BN, STG, CS>;
  static bool attr_set = false;
  static int n_sm = 0;
  if (!attr_set) {
    MK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)gemm_persistent_smem_bytes<BN, STG, CS>()));
    int dev = 0;
    MK(cudaGetDevice(&dev));
    MK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    attr_set = true;
  }
  const int tiles_m = (M + 127) / 128, tiles = tiles_m * ((N + BN - 1) / BN);
  const int grid = std::max(1, std::min(tiles, n_sm));
  kern<<<grid, 32 * (4 * CS + 2), gemm_persistent_smem_bytes<BN, STG, CS>(), st>>>(ta, tb, K, tiles_m, tiles, ep);
  MK(cudaGetLastError());
}

int round8(int x) { return (x + 7) & ~7; }

}  // namespace

struct nrto_mlp {
  int L = 0;                       // layers
  std::vector<int> dims;           // L+1 widths
  int in_pad = 0;                  // input width rounded up to 8
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  long long n_params = 0;
  std::vector<long long> woff, boff;
  std::vector<void*> allocs;
  float *theta = nullptr, *grad = nullptr, *mom1 = nullptr, *mom2 = nullptr;
  std::vector<bf16*> Wt, Wkn;      // per layer
  std::vector<int> ldt;            // leading dim of Wt (input width, padded)
  bf16* X = nullptr;               // [B][in_pad]
  std::vector<bf16*> H;            // H[l], l = 1..L-1: [B][dims[l]]
  std::vector<float*> Z;           // Z[l], l = 1..L-1
  float* Y = nullptr;              // [B][dims[L]]
  std::vector<bf16*> dZ;           // dZ[l], l = 1..L: [B][dims[l]]
  bf16 *tA = nullptr, *tB = nullptr;   // transposes
  float *stage_in = nullptr, *stage_t = nullptr, *stage_m = nullptr;
  double* d_loss = nullptr;
  int* d_err = nullptr;
  long long adam_t = 0;
  long long launches = 0;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gemm_events;   // around each GEMM launch
  double gemm_flops = 0.0;                                         // 2·M·N·K of the timed launches

  template <int BN, int EPI, int STG = GEMM_STAGES>
  void gemm(const bf16* A, long long lda, const bf16* B, long long ldb, int M, int N, int K, const EpiArgs& ep) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (profiling) {
      MK(cudaEventCreate(&e0));
      MK(cudaEventCreate(&e1));
      MK(cudaEventRecord(e0, stream));
    }
    launch_gemm<BN, EPI, STG>(stream, A, lda, B, ldb, M, N, K, ep);
    if (profiling) {
      MK(cudaEventRecord(e1, stream));
      gemm_events.push_back({e0, e1});
      gemm_flops += 2.0 * M * N * K;
    }
  }

  void gemm_out(const bf16* A, long long lda, const bf16* B, long long ldb, int M, int N, int K, const EpiArgs& ep) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (profiling) {
      MK(cudaEventCreate(&e0));
      MK(cudaEventCreate(&e1));
      MK(cudaEventRecord(e0, stream));
    }
    launch_gemm_persistent<256, 3, NRTO_GEMM_CS>(stream, A, lda, B, ldb, M, N, K, ep);
    if (profiling) {
      MK(cudaEventRecord(e1, stream));
      gemm_events.push_back({e0, e1});
      gemm_flops += 2.0 * M * N * K;
    }
  }

  template <typename T>
  T* dalloc(size_t count) {
    void* p = nullptr;
    MK(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
    allocs.push_back(p);
    MK(cudaMemsetAsync(p, 0, std::max<size_t>(count, 1) * sizeof(T), stream));
    return static_cast<T*>(p);
  }
  ~nrto_mlp() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& ev : gemm_events) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
    for (void* p : allocs) cudaFree(p);
  }
  void refresh_bf16() {
    for (int l = 0; l < L; ++l) {
      k_weights_bf16<<<512, 256, 0, stream>>>(theta + woff[l], dims[l + 1], dims[l], Wt[l], ldt[l], l > 0 ? Wkn[l] : nullptr);
      MK(cudaGetLastError());
      ++launches;
    }
  }
  void check_err() {
    int e = 0;
    MK(cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    MK(cudaStreamSynchronize(stream));
    if (e) mfail(NRTO_ERR_TIMEOUT, "a GEMM pipeline wait gave up");
  }
  // forward on the batch already in X (bf16)
  void forward(int B) {
    for (int l = 0; l < L; ++l) {
      const bf16* A = (l == 0) ? X : H[l];
      const long long lda = (l == 0) ? in_pad : dims[l];
      const int K = (l == 0) ? in_pad : dims[l];
      EpiArgs ep{};
      ep.M = B; ep.N = dims[l + 1]; ep.bias = theta + boff[l]; ep.err = d_err;
      if (l < L - 1) {
        ep.out_f32 = Z[l + 1]; ep.ld_f32 = dims[l + 1]; ep.out_bf16 = H[l + 1]; ep.ld_bf16 = dims[l + 1];
        gemm<64, EPI_BIAS_GELU>(A, lda, Wt[l], ldt[l], B, dims[l + 1], K, ep);
      } else {
        ep.out_f32 = Y; ep.ld_f32 = dims[L];
        // the output layer (wide N, short K): the persistent GEMM, epilogue overlapped with the MMAs
        gemm_out(A, lda, Wt[l], ldt[l], B, dims[l + 1], K, ep);
      }
      ++launches;
    }
  }
  // gradients of the masked MSE for the batch in X with targets/mask staged; returns Σ mask·(y-t)²
  void backward(int B, double inv_n) {
    const long long ny = (long long)B * dims[L];
    MK(cudaMemsetAsync(d_loss, 0, sizeof(double), stream));
    k_mse_grad<<<1024, 256, 0, stream>>>(Y, stage_t, stage_m, ny, inv_n, dZ[L], d_loss);
    MK(cudaGetLastError());
    ++launches;
    for (int l = L - 1; l >= 0; --l) {
      const int dout = dims[l + 1], din = dims[l];
      // dW_l = dZ_{l+1}ᵀ · H_l
      dim3 tb(32, 8);
      k_transpose_bf16<<<dim3((dout + 31) / 32, (B + 31) / 32), tb, 0, stream>>>(dZ[l + 1], B, dout, dout, tA, B);
      const bf16* Hl = (l == 0) ? X : H[l];
      const int hw = (l == 0) ? in_pad : din;
      k_transpose_bf16<<<dim3((hw + 31) / 32, (B + 31) / 32), tb, 0, stream>>>(Hl, B, hw, hw, tB, B);
      MK(cudaGetLastError());
      EpiArgs ew{};
      ew.M = dout; ew.N = din; ew.out_f32 = grad + woff[l]; ew.ld_f32 = din; ew.err = d_err;
      gemm<64, EPI_F32>(tA, B, tB, B, dout, din, B, ew);
      k_colsum_bf16<<<(dout + 255) / 256, 256, 0, stream>>>(dZ[l + 1], B, dout, dout, grad + boff[l]);
      MK(cudaGetLastError());
      launches += 4;
      if (l > 0) {
        // dZ_l = (dZ_{l+1} · W_l) ⊙ gelu'(Z_l)
        EpiArgs eb{};
        eb.M = B; eb.N = din; eb.out_bf16 = dZ[l]; eb.ld_bf16 = din; eb.zin = Z[l]; eb.ld_zin = din; eb.err = d_err;
        gemm<64, EPI_GELU_BWD>(dZ[l + 1], dout, Wkn[l], dout, B, din, dout, eb);
        ++launches;
      }
    }
  }
};

void nrto_mlp_set_error_internal(const MlpError& e) { nrto_internal_set_error(e.msg); }

extern "C" {

nrto_status nrto_mlp_create(const int* dims, int n_dims, int max_batch, void* stream, nrto_mlp_t* out) {
  nrto_mlp* m = nullptr;
  try {
    if (!dims || n_dims < 2 || !out) mfail(NRTO_ERR_INVALID, "dims (>= 2 widths) and out are required");
    if (max_batch < 8 || max_batch % 8 != 0) mfail(NRTO_ERR_INVALID, "max_batch must be a positive multiple of 8");
    for (int i = 0; i < n_dims; ++i)
      if (dims[i] < 1 || dims[i] > 65536) mfail(NRTO_ERR_INVALID, "layer widths must be in [1, 65536]");
    for (int i = 1; i < n_dims; ++i)
      if (dims[i] % 8 != 0) mfail(NRTO_ERR_INVALID, "hidden and output widths must be multiples of 8");
    m = new nrto_mlp();
    m->stream = static_cast<cudaStream_t>(stream);
    m->L = n_dims - 1;
    m->dims.assign(dims, dims + n_dims);
    m->in_pad = round8(dims[0]);
    m->max_batch = max_batch;
    long long o = 0;
    for (int l = 0; l < m->L; ++l) {
      m->woff.push_back(o);
      o += (long long)dims[l + 1] * dims[l];
      m->boff.push_back(o);
      o += dims[l + 1];
    }
    m->n_params = o;
    m->theta = m->dalloc<float>(o);
    m->grad = m->dalloc<float>(o);
    m->mom1 = m->dalloc<float>(o);
    m->mom2 = m->dalloc<float>(o);
    int maxw = m->in_pad;
    for (int l = 0; l < m->L; ++l) {
      const int ld = (l == 0) ? m->in_pad : dims[l];
      m->ldt.push_back(ld);
      m->Wt.push_back(m->dalloc<bf16>((size_t)dims[l + 1] * ld));
      m->Wkn.push_back(l > 0 ? m->dalloc<bf16>((size_t)dims[l] * dims[l + 1]) : nullptr);
      maxw = std::max(maxw, dims[l + 1]);
    }
    const size_t B = max_batch;
    m->X = m->dalloc<bf16>(B * m->in_pad);
    m->H.assign(m->L + 1, nullptr);
    m->Z.assign(m->L + 1, nullptr);
    m->dZ.assign(m->L + 1, nullptr);
    for (int l = 1; l < m->L; ++l) {
      m->H[l] = m->dalloc<bf16>(B * dims[l]);
      m->Z[l] = m->dalloc<float>(B * dims[l]);
    }
    for (int l = 1; l <= m->L; ++l) m->dZ[l] = m->dalloc<bf16>(B * dims[l]);
    m->Y = m->dalloc<float>(B * dims[m->L]);
    m->tA = m->dalloc<bf16>(B * maxw);
    m->tB = m->dalloc<bf16>(B * maxw);
    m->stage_in = m->dalloc<float>(B * dims[0]);
    m->stage_t = m->dalloc<float>(B * dims[m->L]);
    m->stage_m = m->dalloc<float>(B * dims[m->L]);
    m->d_loss = m->dalloc<double>(1);
    m->d_err = m->dalloc<int>(1);
    MK(cudaStreamSynchronize(m->stream));
    *out = m;
    return NRTO_OK;
  } catch (const MlpError& e) {
    delete m;
    nrto_mlp_set_error_internal(e);
    return e.st;
  }
}

nrto_status nrto_mlp_destroy(nrto_mlp_t m) {
  delete m;
  return NRTO_OK;
}

long long nrto_mlp_num_params(nrto_mlp_t m) { return m ? m->n_params : -1; }

nrto_status nrto_mlp_set_params(nrto_mlp_t m, const float* params) {
  try {
    if (!m || !params) mfail(NRTO_ERR_INVALID, "null argument");
    for (long long i = 0; i < m->n_params; ++i)
      if (!std::isfinite(params[i])) mfail(NRTO_ERR_NUMERIC, "parameters not finite");
    MK(cudaMemcpyAsync(m->theta, params, sizeof(float) * m->n_params, cudaMemcpyHostToDevice, m->stream));
    MK(cudaMemsetAsync(m->mom1, 0, sizeof(float) * m->n_params, m->stream));
    MK(cudaMemsetAsync(m->mom2, 0, sizeof(float) * m->n_params, m->stream));
    m->adam_t = 0;
    m->refresh_bf16();
    MK(cudaStreamSynchronize(m->stream));
    return NRTO_OK;
  } catch (const MlpError& e) {
    nrto_mlp_set_error_internal(e);
    return e.st;
  }
}

nrto_status nrto_mlp_get_params(nrto_mlp_t m, float* params) {
  try {
    if (!m || !params) mfail(NRTO_ERR_INVALID, "null argument");
    MK(cudaMemcpyAsync(params, m->theta, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    return NRTO_OK;
  } catch (const MlpError& e) {
    nrto_mlp_set_error_internal(e);
    return e.st;
  }
}

nrto_status nrto_mlp_forward(nrto_mlp_t m, const float* x, int batch, float* y) {
  try {
    if (!m || !x || !y) mfail(NRTO_ERR_INVALID, "null argument");
    if (batch < 1 || batch > m->max_batch) mfail(NRTO_ERR_INVALID, "batch out of range");
    MK(cudaMemcpyAsync(m->stage_in, x, sizeof(float) * (size_t)batch * m->dims[0], cudaMemcpyHostToDevice, m->stream));
    k_to_bf16_pad<<<512, 256, 0, m->stream>>>(m->stage_in, batch, m->dims[0], m->X, m->in_pad);
    MK(cudaGetLastError());
    ++m->launches;
    m->forward(batch);
    MK(cudaMemcpyAsync(y, m->Y, sizeof(float) * (size_t)batch * m->dims[m->L], cudaMemcpyDeviceToHost, m->stream));
    m->check_err();
    return NRTO_OK;
  } catch (const MlpError& e) {
    nrto_mlp_set_error_internal(e);
    return e.st;
  }
}

nrto_status nrto_mlp_train_step(nrto_mlp_t m, const float* x, const float* target, const float* mask, int batch,
                                float lr, double* loss, float* grads) {
  try {
    if (!m || !x || !target || !mask) mfail(NRTO_ERR_INVALID, "null argument");
    if (batch < 8 || batch > m->max_batch || batch % 8 != 0) mfail(NRTO_ERR_INVALID, "batch must be a multiple of 8 within max_batch");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) mfail(NRTO_ERR_INVALID, "learning rate must be finite and >= 0");
    const size_t ny = (size_t)batch * m->dims[m->L];
    double n_mask = 0.0;
    for (size_t q = 0; q < ny; ++q) n_mask += mask[q];
    if (!(n_mask > 0.0)) mfail(NRTO_ERR_INVALID, "mask selects no output");
    MK(cudaMemcpyAsync(m->stage_in, x, sizeof(float) * (size_t)batch * m->dims[0], cudaMemcpyHostToDevice, m->stream));
    MK(cudaMemcpyAsync(m->stage_t, target, sizeof(float) * ny, cudaMemcpyHostToDevice, m->stream));
    MK(cudaMemcpyAsync(m->stage_m, mask, sizeof(float) * ny, cudaMemcpyHostToDevice, m->stream));
    k_to_bf16_pad<<<512, 256, 0, m->stream>>>(m->stage_in, batch, m->dims[0], m->X, m->in_pad);
    MK(cudaGetLastError());
    ++m->launches;
    m->forward(batch);
    m->backward(batch, 1.0 / n_mask);
    if (grads) MK(cudaMemcpyAsync(grads, m->grad, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, m->stream));
    double lsum = 0.0;
    MK(cudaMemcpyAsync(&lsum, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if (lr > 0.0f) {
      m->adam_t += 1;
      const float c1 = (float)(1.0 - std::pow(0.9, (double)m->adam_t));
      const float c2 = (float)(1.0 - std::pow(0.999, (double)m->adam_t));
      k_adam<<<1024, 256, 0, m->stream>>>(m->theta, m->grad, m->mom1, m->mom2, m->n_params, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
      MK(cudaGetLastError());
      ++m->launches;
      m->refresh_bf16();
    }
    m->check_err();
    if (loss) *loss = lsum / n_mask;
    return NRTO_OK;
  } catch (const MlpError& e) {
    nrto_mlp_set_error_internal(e);
    return e.st;
  }
}

long long nrto_mlp_kernel_launches(nrto_mlp_t m) { return m ? m->launches : -1; }

}  // extern "C"

// For the library's own use (warm start from the network): forward of a host batch with the output
// left on the device (stream-ordered on the network's stream).  Returns null on error (message set).
const float* nrto_mlp_internal_forward_device(nrto_mlp_t m, const float* x, int batch, int* out_dim,
                                              cudaStream_t* stream) {
  try {
    if (!m || !x) mfail(NRTO_ERR_INVALID, "null argument");
    if (batch < 1 || batch > m->max_batch) mfail(NRTO_ERR_INVALID, "batch exceeds the network's max_batch");
    MK(cudaMemcpyAsync(m->stage_in, x, sizeof(float) * (size_t)batch * m->dims[0], cudaMemcpyHostToDevice, m->stream));
    k_to_bf16_pad<<<512, 256, 0, m->stream>>>(m->stage_in, batch, m->dims[0], m->X, m->in_pad);
    MK(cudaGetLastError());
    ++m->launches;
    m->forward(batch);
    *out_dim = m->dims[m->L];
    *stream = m->stream;
    return m->Y;
  } catch (const MlpError& e) {
    nrto_mlp_set_error_internal(e);
    return nullptr;
  }
}

extern "C" {

nrto_status nrto_mlp_profile(nrto_mlp_t m, int enable, double* gemm_ms, double* gemm_flops, long long* gemm_launches) {
  try {
    if (!m) mfail(NRTO_ERR_INVALID, "null network");
    double ms = 0.0;
    if (!m->gemm_events.empty()) {
      MK(cudaStreamSynchronize(m->stream));
      for (auto& ev : m->gemm_events) {
        float t = 0.f;
        MK(cudaEventElapsedTime(&t, ev.first, ev.second));
        ms += t;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
      }
    }
    if (gemm_ms) *gemm_ms = ms;
    if (gemm_flops) *gemm_flops = m->gemm_flops;
    if (gemm_launches) *gemm_launches = (long long)m->gemm_events.size();
    m->gemm_events.clear();
    m->gemm_flops = 0.0;
    m->profiling = enable != 0;
    return NRTO_OK;
  } catch (const MlpError& e) {
    nrto_mlp_set_error_internal(e);
    return e.st;
  }
}

}  // extern "C"
