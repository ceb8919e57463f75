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
// line order, as the next pass's A operand in shared memory.  Thread t of the CTA owns row t
// in every pass (tile t / 128, lane t % 128), so the only exchange between threads is that
// transpose.  The matrix of the next pass is brought into the other of two B buffers by a bulk
// (TMA) copy while the current pass runs.
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
  // CTAs per SM the registers are sized for: one at N = 24 (its operands take most of the
  // shared memory), two below, so that one CTA's conversions overlap the other's MMAs
  static constexpr int MINB = N >= 24 ? 1 : 2;
  static constexpr int A_PART = 128 * K;  // BF16 values of one tile of one split term
  static constexpr int B_PART = NN * K;   // BF16 values of one split term of a matrix
  static constexpr int A_ELEMS = TILES * 3 * A_PART;
  static constexpr int B_ELEMS = 3 * B_PART;  // one matrix image: three split terms
  static constexpr int REGION = pow2_at_least(TILES * NN);  // TMEM columns of one volume
  static constexpr int TMEM_COLS = 2 * REGION;              // pass output + product accumulator
  static constexpr size_t SMEM = size_t(A_ELEMS + 2 * B_ELEMS) * 2;  // A + two matrix buffers
  static constexpr uint32_t SBO = 16u * K;  // bytes between 8-row groups of an operand
  static constexpr uint32_t LBO = 128u;     // bytes between 8-column groups
  static constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, NN);
  static_assert(K % 16 == 0, "the line length must fill whole MMA K steps");
  static_assert(N % 8 == 0, "the line orders work on octets of each coordinate");
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

// ---- line orders --------------------------------------------------------------------------
// Each pass stores its lines in an order of its own: row r of the pass (TMEM lane r % 128 of tile
// r / 128, owned by thread r) holds one line.  The orders are chosen so that the transposing
// stores of every conversion hit 32 distinct shared-memory banks per warp.  The 4-byte store of
// (row R, column 2u) lands in bank 4 (R % 8) + u % 4, so a warp's 32 lanes must cover the 8
// values of R % 8 of the target rows times 4 values of u % 4.
//   kPX  (x pass of an x, y, z transform), lines (y, z): a warp is 4 y x 8 z, row % 8 free;
//   kPY  (y pass after kPX), lines (x, z): row % 8 = z % 8 (the x -> y stores), and a warp holds
//        8 values of x % 8, each with 4 values of z % 4 (the y -> z stores);
//   kPZ  (z pass, both orders), lines (x, y): row % 8 = x % 8;
//   kPY2 (y pass after kPZ in a z, y, x transform), lines (x, z): row % 8 = x % 8, and a warp
//        holds 8 values of z % 8, each with 4 values of x % 4;
//   kPX2 (x pass after kPY2), lines (y, z): row % 8 = z % 8.
// The middle orders pair x (or z) with the parity bit of the other coordinate's half-octet so
// that both conditions hold at once.  N is a multiple of 8.
enum PassOrder { kPX = 0, kPY = 1, kPZ = 2, kPY2 = 3, kPX2 = 4 };

template <int P> struct PassAxis { static constexpr int value = (P == kPX || P == kPX2) ? 0 : (P == kPZ ? 2 : 1); };

// row of the line through (x, y, z) along the pass's axis (the axis coordinate is ignored)
template <int N, int P>
__device__ __forceinline__ int row_of(int x, int y, int z) {
  constexpr int E = N >> 3;
  if constexpr (P == kPX) return (((y >> 2) * E + (z >> 3)) << 5) + ((z & 7) << 2) + (y & 3);
  if constexpr (P == kPY) return ((((x >> 3) * E + (z >> 3)) * 2 + (((z & 7) >> 2) ^ (x & 1))) << 5) + (((x & 7) >> 1) << 3) + (z & 7);
  if constexpr (P == kPZ) return (((x >> 3) * N + y) << 3) + (x & 7);
  if constexpr (P == kPY2) return ((((z >> 3) * E + (x >> 3)) * 2 + (((x & 7) >> 2) ^ (z & 1))) << 5) + (((z & 7) >> 1) << 3) + (x & 7);
  return (((z >> 3) * N + y) << 3) + (z & 7);  // kPX2
}
// the line of row r: sets the two coordinates that are not the pass's axis
template <int N, int P>
__device__ __forceinline__ void line_of(int r, int (&c)[3]) {
  constexpr int E = N >> 3;
  if constexpr (P == kPX) {
    const int blk = r >> 5;
    c[1] = ((blk / E) << 2) + (r & 3);
    c[2] = ((blk % E) << 3) + ((r >> 2) & 7);
  } else if constexpr (P == kPY) {
    const int zl = r & 7, g = (r >> 3) & 3, par = (r >> 5) & 1, blk = r >> 6;
    c[0] = ((blk / E) << 3) + 2 * g + ((zl >> 2) ^ par);
    c[2] = ((blk % E) << 3) + zl;
  } else if constexpr (P == kPZ) {
    const int q = r >> 3;
    c[0] = ((q / N) << 3) + (r & 7);
    c[1] = q % N;
  } else if constexpr (P == kPY2) {
    const int xl = r & 7, g = (r >> 3) & 3, par = (r >> 5) & 1, blk = r >> 6;
    c[2] = ((blk / E) << 3) + 2 * g + ((xl >> 2) ^ par);
    c[0] = ((blk % E) << 3) + xl;
  } else {
    const int q = r >> 3;
    c[2] = ((q / N) << 3) + (r & 7);
    c[1] = q % N;
  }
}

// The MMAs of one pass (one thread): for every tile of 128 rows, the six split-term products
// over the K steps, accumulated into that tile's columns of tensor memory.  da / db describe the
// starts of the A operand and of the current matrix buffer; each MMA adds a compile-time byte
// offset (>> 4) to their address fields (the operands lie below 256 KB: no carry out).  Kept
// out of line: one copy of the unrolled sequence serves every pass.
template <int N>
__device__ __noinline__ void issue_pass_mmas(uint64_t da, uint64_t db, uint32_t tmem) {
  using G = GemmGeo<N>;
#pragma unroll
  for (int tile = 0; tile < G::TILES; ++tile) {
    const uint32_t d = tmem + uint32_t(tile * G::NN);
#pragma unroll
    for (int pr = 0; pr < 6; ++pr) {
#pragma unroll
      for (int ks = 0; ks < G::K / 16; ++ks) {
        const uint32_t oa = (uint32_t((tile * 3 + kProdA[pr]) * G::A_PART) * 2u + uint32_t(ks) * 256u) >> 4;
        const uint32_t ob = (uint32_t(kProdB[pr] * G::B_PART) * 2u + uint32_t(ks) * 256u) >> 4;
        tc::mma_bf16(d, da + oa, db + ob, G::IDESC, (pr | ks) != 0 ? 1u : 0u);
      }
    }
  }
}

// Shared state of one CTA running DFT passes.
template <int N>
struct GemmCta {
  using G = GemmGeo<N>;
  uint16_t* A;         // [TILES][3][A_PART]
  uint16_t* B;         // [2][3][B_PART]: matrix images, double-buffered
  uint64_t* bar;       // MMA completion barrier
  uint64_t* bbar;      // [2] bulk-copy barriers of the two matrix buffers
  uint32_t tmem;       // base address of the CTA's tensor memory
  uint32_t phase;      // parity of the MMA barrier's next completion
  uint32_t bphase;     // bit i: parity of matrix buffer i's next completion
  int bsel;            // matrix buffer of the next pass
  int* abort_flag;     // shared: set when a bounded wait gave up
  unsigned* status;    // global: device status word (set on timeout)

  // this thread's lane in the pass output (its row t): tile t / 128, lane t % 128
  __device__ __forceinline__ uint32_t lane_addr(int t, int region) const {
    const int tile = t >> 7, lane = t & 127;
    return tmem + (uint32_t(lane & ~31) << 16) + uint32_t(region * G::REGION + tile * G::NN);
  }
  // store one complex value, split, at (row R, column 2u) of the A operand
  __device__ __forceinline__ void put(int R, int u, float re, float im) const {
    uint32_t w0, w1, w2;
    split3(re, im, w0, w1, w2);
    uint16_t* base = A + size_t(R >> 7) * 3 * G::A_PART + op_index(R & 127, 2 * u, G::K);
    *reinterpret_cast<uint32_t*>(base) = w0;
    *reinterpret_cast<uint32_t*>(base + G::A_PART) = w1;
    *reinterpret_cast<uint32_t*>(base + 2 * G::A_PART) = w2;
  }
  // store the whole row R of the A operand from 2N floats (re, im interleaved, in order)
  __device__ __forceinline__ void put_row(int R, const float* v) const {
    uint16_t* base = A + size_t(R >> 7) * 3 * G::A_PART;
#pragma unroll
    for (int c = 0; c < G::K / 8; ++c) {  // 4 complex values = 16 bytes per split term
      uint32_t w[3][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) split3(v[8 * c + 2 * j], v[8 * c + 2 * j + 1], w[0][j], w[1][j], w[2][j]);
      const int o = op_index(R & 127, 8 * c, G::K);
#pragma unroll
      for (int part = 0; part < 3; ++part)
        *reinterpret_cast<uint4*>(base + part * G::A_PART + o) = make_uint4(w[part][0], w[part][1], w[part][2], w[part][3]);
    }
  }
  // thread 0: start the bulk copy of a matrix image into the next pass's buffer (its previous
  // reader, the pass before the last, has completed)
  __device__ __forceinline__ void prefetch_matrix(const uint16_t* img, int tid) const {
    if (tid == 0) {
      constexpr uint32_t bytes = uint32_t(G::B_ELEMS) * 2u;
      tc::mbar_expect_tx(&bbar[bsel], bytes);
      tc::bulk_g2s(B + size_t(bsel) * G::B_ELEMS, img, bytes, &bbar[bsel]);
    }
  }
  // make the A operand visible to the tensor core, issue the pass's MMAs (thread 0, after the
  // matrix copy into buffer bsel has landed; then the copy of `next` into the other buffer
  // starts) and wait for them; returns false when a wait gave up (the CTA then stops)
  __device__ __forceinline__ bool mma_pass(int tid, const uint16_t* next) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      bool ok = tc::mbar_wait_bounded(&bbar[bsel], (bphase >> bsel) & 1u, 2000000000LL);
      if (ok) {
        issue_pass_mmas<N>(tc::smem_desc(tc::smem_addr(A), G::LBO, G::SBO),
                           tc::smem_desc(tc::smem_addr(B + size_t(bsel) * G::B_ELEMS), G::LBO, G::SBO), tmem);
        tc::mma_commit(bar);
      } else {
        *abort_flag = 1;
        if (status) atomicOr(status, 1u);
      }
    }
    bphase ^= 1u << bsel;
    bsel ^= 1;
    if (next) prefetch_matrix(next, tid);
    // about one second at the GB300's clock; a CTA whose matrix copy gave up skips the wait
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

// Transpose the previous pass's output (TMEM region 0, pass order POLD) into the A operand of
// the next pass (order PNEW).  Thread t owns row t of the previous pass.
template <int N, int POLD, int PNEW>
__device__ __forceinline__ void convert_pass(const GemmCta<N>& cta, int t) {
  using G = GemmGeo<N>;
  constexpr int AOLD = PassAxis<POLD>::value, ANEW = PassAxis<PNEW>::value;
  if ((t & ~31) >= G::N2) return;  // a warp of padding rows (warp-uniform)
  int co[3];
  line_of<N, POLD>(t, co);
  const uint32_t ta = cta.lane_addr(t, 0);
#pragma unroll 1
  for (int ch = 0; ch < G::NN / 16; ++ch) {
    float v[16];
    tc::tmem_ld16(ta + uint32_t(16 * ch), v);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      co[AOLD] = 8 * ch + j;
      cta.put(row_of<N, PNEW>(co[0], co[1], co[2]), co[ANEW], v[2 * j], v[2 * j + 1]);
    }
  }
}

}  // namespace dgfs
