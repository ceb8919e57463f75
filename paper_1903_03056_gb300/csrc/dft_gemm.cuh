// Three-dimensional DFTs as dense contractions on the tensor cores (tcgen05), split-BF16
// arithmetic with FP32 accumulation: the building block of the DGFS_BF16X3 collision path.
//
// A 3D transform of an N^3 complex volume is three passes, one per axis.  A pass is the matrix
// product D = X W^T over the N^2 lines of the volume along that axis: X [lines][2N] holds each
// line's N complex inputs as interleaved (re, im), W [2N][2N] is the real form of the line
// transform (with the per-axis phase factor of the shifted transforms of Sec. 4 folded into its
// columns), D [lines][2N] the line's outputs.  Lines are the MMA's M dimension in tiles of 128
// (tensor-memory lanes), the outputs its N dimension (2N columns), the inputs its K dimension
// (2N, in steps of 16).
//
// Precision: every FP32 value x is split exactly into three BF16 terms x0 + x1 + x2 (each the
// BF16 rounding of what the previous terms leave); the same for W.  The six products
// x0 w0, x0 w1, x1 w0, x0 w2, x1 w1, x2 w0 are accumulated in FP32 in tensor memory; the three
// dropped ones are below 2^-23 of |x w|, the same order as FP32 rounding.
//
// Data movement per pass: the pass's output D stays in tensor memory; each thread reads its own
// lane (line) back with tcgen05.ld, splits it and writes it, transposed into the next pass's
// line order, as the next pass's A operand in shared memory.  Thread t of the CTA owns line t
// in every pass (tile t / 128, lane t % 128), so the only exchange between threads is that
// transpose.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tcgen05.cuh"

namespace dgfs {

constexpr int pow2_at_least(int v, int p = 32) { return p >= v ? p : pow2_at_least(v, 2 * p); }

template <int N>
struct GemmGeo {
  static constexpr int N2 = N * N;
  static constexpr int N3 = N * N * N;
  static constexpr int K = 2 * N;    // real inputs of a line (re, im interleaved)
  static constexpr int NN = 2 * N;   // real outputs of a line
  static constexpr int TILES = (N2 + 127) / 128;
  static constexpr int THREADS = 128 * TILES;
  static constexpr int A_PART = 128 * K;  // BF16 values of one tile of one split term
  static constexpr int B_PART = NN * K;   // BF16 values of one split term of a matrix
  static constexpr int A_ELEMS = TILES * 3 * A_PART;
  static constexpr int B_ELEMS = 3 * B_PART;  // one matrix image: three split terms
  static constexpr int REGION = pow2_at_least(TILES * NN);  // TMEM columns of one volume
  static constexpr int TMEM_COLS = 2 * REGION;              // pass output + product accumulator
  static constexpr size_t SMEM = size_t(A_ELEMS + B_ELEMS) * 2;
  static constexpr uint32_t SBO = 16u * K;  // bytes between 8-row groups of an operand
  static constexpr uint32_t LBO = 128u;     // bytes between 8-column groups
  static constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, NN);
  static_assert(K % 16 == 0, "the line length must fill whole MMA K steps");
  static_assert(N2 % 32 == 0, "lines must fill whole warps");
};

// index (in 16-bit units) of element (r, k) of an operand with K columns (canonical K-major
// layout without swizzle; 8 x 8 core matrices of 128 bytes)
__host__ __device__ constexpr int op_index(int r, int k, int K) {
  return (r >> 3) * (K >> 3) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// the split term products kept: (term of the data, term of the matrix), smallest first.  The
// tensor core's FP32 accumulator does not round to nearest when it adds a product to a larger
// partial sum, so the 2^-16 and 2^-8 terms are summed among themselves before the leading
// product joins them (measured: the 3D transform's error fell from 1.9e-6 to 1.7e-7 of max |y|).
__device__ constexpr int kProdA[6] = {1, 0, 2, 0, 1, 0};
__device__ constexpr int kProdB[6] = {1, 2, 0, 1, 0, 0};

// (re, im) -> three BF16 pairs whose sum is (re, im) exactly
__device__ __forceinline__ void split3(float re, float im, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  const __nv_bfloat162 h0 = __floats2bfloat162_rn(re, im);
  const float2 f0 = __bfloat1622float2(h0);
  const float r1 = re - f0.x, i1 = im - f0.y;
  const __nv_bfloat162 h1 = __floats2bfloat162_rn(r1, i1);
  const float2 f1 = __bfloat1622float2(h1);
  const __nv_bfloat162 h2 = __floats2bfloat162_rn(r1 - f1.x, i1 - f1.y);
  w0 = *reinterpret_cast<const uint32_t*>(&h0);
  w1 = *reinterpret_cast<const uint32_t*>(&h1);
  w2 = *reinterpret_cast<const uint32_t*>(&h2);
}

// Shared state of one CTA running DFT passes.
template <int N>
struct GemmCta {
  using G = GemmGeo<N>;
  uint16_t* A;         // [TILES][3][A_PART]
  uint16_t* B;         // [3][B_PART]
  uint64_t* bar;       // MMA completion barrier
  uint32_t tmem;       // base address of the CTA's tensor memory
  uint32_t phase;      // parity of the barrier's next completion
  int* abort_flag;     // shared: set when a bounded wait gave up
  unsigned* status;    // global: device status word (set on timeout)

  // this thread's lane in the pass output (its line t): tile t / 128, lane t % 128
  __device__ __forceinline__ uint32_t lane_addr(int t, int region) const {
    const int tile = t >> 7, lane = t & 127;
    return tmem + (uint32_t(lane & ~31) << 16) + uint32_t(region * G::REGION + tile * G::NN);
  }
  // store one complex value, split, at (row L, column 2u) of the A operand
  __device__ __forceinline__ void put(int L, int u, float re, float im) const {
    uint32_t w0, w1, w2;
    split3(re, im, w0, w1, w2);
    uint16_t* base = A + size_t(L >> 7) * 3 * G::A_PART + op_index(L & 127, 2 * u, G::K);
    *reinterpret_cast<uint32_t*>(base) = w0;
    *reinterpret_cast<uint32_t*>(base + G::A_PART) = w1;
    *reinterpret_cast<uint32_t*>(base + 2 * G::A_PART) = w2;
  }
  // store the whole row L of the A operand from 2N floats (re, im interleaved, in order)
  __device__ __forceinline__ void put_row(int L, const float* v) const {
    uint16_t* base = A + size_t(L >> 7) * 3 * G::A_PART;
#pragma unroll
    for (int c = 0; c < G::K / 8; ++c) {  // 4 complex values = 16 bytes per split term
      uint32_t w[3][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) split3(v[8 * c + 2 * j], v[8 * c + 2 * j + 1], w[0][j], w[1][j], w[2][j]);
      const int o = op_index(L & 127, 8 * c, G::K);
#pragma unroll
      for (int part = 0; part < 3; ++part)
        *reinterpret_cast<uint4*>(base + part * G::A_PART + o) = make_uint4(w[part][0], w[part][1], w[part][2], w[part][3]);
    }
  }
  // copy one matrix image (3 split terms) from global memory into the B operand
  __device__ __forceinline__ void load_matrix(const uint16_t* img, int tid) const {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(B);
    for (int i = tid; i < G::B_ELEMS / 8; i += G::THREADS) dst[i] = __ldg(src + i);
  }
  // make the operands visible to the tensor core, issue the pass's MMAs (thread 0) and wait
  // for them; returns false when the wait gave up (the CTA then stops)
  __device__ __forceinline__ bool mma_pass(int tid) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
#pragma unroll 1
      for (int tile = 0; tile < G::TILES; ++tile) {
        const uint32_t d = tmem + uint32_t(tile * G::NN);
        uint32_t acc = 0;
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
#pragma unroll
          for (int ks = 0; ks < G::K / 16; ++ks) {
            const uint32_t aa = a0 + uint32_t((tile * 3 + kProdA[pr]) * G::A_PART) * 2u + uint32_t(ks) * 256u;
            const uint32_t bb = b0 + uint32_t(kProdB[pr] * G::B_PART) * 2u + uint32_t(ks) * 256u;
            tc::mma_bf16(d, tc::smem_desc(aa, G::LBO, G::SBO), tc::smem_desc(bb, G::LBO, G::SBO), G::IDESC, acc);
            acc = 1;
          }
        }
      }
      tc::mma_commit(bar);
    }
    // about one second at the GB300's clock
    const bool ok = tc::mbar_wait_bounded(bar, phase, 2000000000LL);
    phase ^= 1u;
    if (!ok) {
      *abort_flag = 1;
      if (status) atomicOr(status, 1u);
    }
    __syncthreads();
    tc::fence_after_sync();
    return *abort_flag == 0;
  }
};

// pass axis orders: lines of a pass over axis a are the other two axes (b < c), line = b N + c
template <int A>
struct LineAxes {
  static constexpr int b = A == 0 ? 1 : 0;
  static constexpr int c = A == 2 ? 1 : 2;
};

// Transpose the previous pass's output (in TMEM region 0, over axis AOLD) into the A operand of
// the next pass (over axis ANEW).  Thread t owns line t of the previous pass.
template <int N, int AOLD, int ANEW>
__device__ __forceinline__ void convert_pass(const GemmCta<N>& cta, int t) {
  using G = GemmGeo<N>;
  if ((t & ~31) >= G::N2) return;  // a warp of padding lines (warp-uniform)
  int co[3];
  co[LineAxes<AOLD>::b] = t / N;
  co[LineAxes<AOLD>::c] = t % N;
  const uint32_t ta = cta.lane_addr(t, 0);
#pragma unroll 1
  for (int ch = 0; ch < G::NN / 16; ++ch) {
    float v[16];
    tc::tmem_ld16(ta + uint32_t(16 * ch), v);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      co[AOLD] = 8 * ch + j;
      const int L = co[LineAxes<ANEW>::b] * N + co[LineAxes<ANEW>::c];
      cta.put(L, co[ANEW], v[2 * j], v[2 * j + 1]);
    }
  }
}

}  // namespace dgfs
