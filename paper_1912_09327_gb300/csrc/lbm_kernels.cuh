// LBMTau1 D2Q9 stream-and-collide step for sm_103a (Matyka & Dzikowski,
// arXiv:1912.09327, Section 2, Algorithm 1).
//
// What one step computes, for every fluid node O (Eqs. rhotau1, utau1 with
// the equilibrium of Eq. maxwellboltzmann and the wall rule of Eq. feqnoslip):
//   rho'(O) = sum_k f_k,   j'(O) = sum_k c_k f_k,   c_k = -e_k,
//   f_k = f^eq_{c_k}(rho(P), (j(P) + F) / rho(P))   if P = O + e_k is not solid,
//   f_k = w_k rho(O)                                if P is solid.
// Solid and fixed nodes keep their values.
//
// Arithmetic form.  The device stores delta = rho - 1 and j.  With
// Pi = j' j'^T / rho (j' = j + F) the equilibrium of a source P seen along c is
//   f^eq_c = w_c (1 + delta + 3 c.j' + 4.5 c^T Pi c - 1.5 tr Pi),
// so each source contributes a fixed linear combination of six per-node
// quantities (delta, j', Pi) to its nine receivers: the moments-only closed
// form that Section 4 derives by multiplying Eq. (LBMTau1) with the raw-moment
// matrix.  The constant "1" parts sum to exactly 1 (mass) and 0 (momentum),
// so they are dropped.  The momentum is updated in increment form,
//   j'(O) = j(O) + (F + sum_k w_k c_k [3 c_k.(j_P - j_O) + ...]),
// with every j_P - j_O taken as an exact FP32 difference before it is
// weighted, so the O(|j|) part of the sum is never rounded: the result then
// carries one rounding of j per step, the floor set by FP32 storage.  A solid
// source enters with delta_P = delta_O, j'_P = 0 and Pi_P = 0, which is
// Eq. (feqnoslip) in this form.
//
// Kernel structure (HBM-bound stencil; no tensor cores).  A block stacks four
// warp tiles of 30 kC columns x kRows rows.  Lane l holds kC adjacent columns
// (one vector per field), so lanes 1..30 own the outputs and lanes 0 and 31
// carry the one-column halos.  Each warp marches down its tile one source row
// at a time; all per-node arithmetic runs on pairs of adjacent columns of
// that row with the packed FP32 instructions (FADD2 / FMUL2 / FFMA2), in the
// order the vector loads deliver them.  Each source row is read from HBM
// once, turned into per-node quantities once (one reciprocal per node), its
// left/right neighbour columns come from warp shuffles (their sums and
// differences formed column by column), and its contributions
// are added to the output rows it feeds (above, same, below); one output row
// completes per source row and is stored as vectors.  Interior warp
// tiles stream their row windows through a ring of shared-memory stages
// filled by bulk asynchronous copies (cp.async.bulk completing on mbarriers,
// every wait bounded in time), several rows ahead of use; at the domain's
// edges the copies are clipped to the row and a periodic axis's wrapped
// column arrives as one more 16-byte block.  On the last step of an lbm_step call the
// same kernel reduces sum |du|^2, sum |u|^2 and sum delta (FP32 per lane, the
// mass compensated, then FP64 warp shuffles into one partial per warp tile)
// and raises a sticky flag on rho <= 0 or non-finite values.
// The storage type T (FP32, or FP16 / BF16 deviations) only changes loads and
// stores; the arithmetic is FP32 throughout.  A batched kernel runs the same
// tile code, warp by warp, over a work list of many domains' warp tiles.
//
// This header holds the kernels as templates; lbm_step_f32.cu, lbm_step_f16.cu
// and lbm_step_bf16.cu instantiate them for one storage format each (compiled
// in parallel), and lbm_step.cu dispatches between them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include <type_traits>

#include "lbm_step.cuh"

namespace lbmtau1 {
namespace {


constexpr int kLanes = 32;
constexpr int kWarps = kTileWarps;            // warps per block, stacked in y
constexpr int kThreads = kWarps * kLanes;
constexpr unsigned kFull = 0xffffffffu;

// D2Q9 weights (rest 4/9, axis 1/9, diagonal 1/36) and the combinations of
// them that appear in the closed form.
// The density a node receives is the weighted sum of its nine sources'
// densities, so the three weights must sum to exactly one in FP32 as well,
// or every step scales the density deviations by their sum (by 1 + 7.5e-9
// with the nearest FP32 values, which drains a multiphase drop of order-one
// deviations by 1e-5 of its mass in 2000 steps).  4/9 and 1/9 are the
// nearest FP32 values; the diagonal weight is one unit in the last place
// below the nearest value of 1/36 (6.7e-8 relative), which makes
// k4_9 + 4 k1_9 + 4 k1_36 == 1 exactly.
constexpr float k4_9 = 4.0f / 9.0f;
constexpr float k1_9 = 1.0f / 9.0f;
constexpr float k1_36 = 0x1.c71c70p-6f;
static_assert(static_cast<double>(k4_9) + 4.0 * static_cast<double>(k1_9) +
                      4.0 * static_cast<double>(k1_36) == 1.0,
              "D2Q9 weights must sum to one in FP32");
constexpr float k1_12 = 1.0f / 12.0f;  // 3 * (1/36)
constexpr float k1_3 = 1.0f / 3.0f;    // 3 * (1/9)
constexpr float k1_6 = 1.0f / 6.0f;    // 2 * (1/12)

// v mod n in [0, n); one period out (the usual case) costs no division.
__device__ __forceinline__ int64_t wrap_index(int64_t v, int64_t n) {
  v = v < 0 ? v + n : (v >= n ? v - n : v);
  if (v < 0 || v >= n) {
    v %= n;
    if (v < 0) v += n;
  }
  return v;
}

// Packed FP32 arithmetic (sm_100 family FADD2 / FMUL2 / FFMA2): every value
// below is a pair (row r, row r + 1) of the same column.
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
  return __fmul2_rn(a, b);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
// a - b, rounded once (exact when a and b are within a factor of 2)
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

// Storage formats.  All arithmetic is FP32; a 16-bit format stores the
// deviations rho - 1 and j scaled by exact powers of two (FP16: 2^10 and 2^6,
// which keep typical values, |rho - 1| >= 1e-7 and |j| >= 1e-6, out of the
// subnormal range; BF16 has FP32's exponent range and needs none).
template <typename T>
struct Storage;
template <>
struct Storage<float> {
  static constexpr float kD = 1.0f, kJ = 1.0f;
  __device__ static float decode(float v) { return v; }
  __device__ static float encode(float v) { return v; }
};
template <>
struct Storage<__half> {
  static constexpr float kD = 1024.0f, kJ = 64.0f;
  __device__ static float decode(__half v) { return __half2float(v); }
  __device__ static __half encode(float v) { return __float2half_rn(v); }
};
template <>
struct Storage<__nv_bfloat16> {
  static constexpr float kD = 1.0f, kJ = 1.0f;
  __device__ static float decode(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __nv_bfloat16 encode(float v) {
    return __float2bfloat16_rn(v);
  }
};

// kC consecutive elements as one vector load / store.
template <int kC, typename T>
struct Vec {
  static constexpr int kBytes = kC * static_cast<int>(sizeof(T));
  using type = typename std::conditional<
      kBytes == 16, uint4,
      typename std::conditional<kBytes == 8, uint2, unsigned>::type>::type;
};

// Loads kC elements at p (vector-aligned) as kC / 2 column pairs, decoded
// and times `inv`; pair q holds columns 2q and 2q + 1, in the order the
// vector brings them, so no register moves pair them.
template <int kC, typename T>
__device__ __forceinline__ void load_pairs(const T *p, float2 (&o)[kC / 2],
                                           float inv) {
  using V = typename Vec<kC, T>::type;
  union {
    V v;
    T e[kC];
  } u;
  u.v = *reinterpret_cast<const V *>(p);
#pragma unroll
  for (int q = 0; q < kC / 2; ++q) {
    const float2 f = make_float2(Storage<T>::decode(u.e[2 * q]),
                                 Storage<T>::decode(u.e[2 * q + 1]));
    if constexpr (std::is_same<T, float>::value)
      o[q] = f;
    else
      o[q] = __fmul2_rn(f, make_float2(inv, inv));
  }
}

// Encodes kC / 2 column pairs times `scale` and stores them as one vector.
template <int kC, typename T>
__device__ __forceinline__ void store_pairs(T *p, const float2 (&v)[kC / 2],
                                            float scale) {
  using V = typename Vec<kC, T>::type;
  union {
    V v;
    T e[kC];
  } u;
#pragma unroll
  for (int q = 0; q < kC / 2; ++q) {
    const float2 f = std::is_same<T, float>::value
                         ? v[q]
                         : __fmul2_rn(v[q], make_float2(scale, scale));
    u.e[2 * q] = Storage<T>::encode(f.x);
    u.e[2 * q + 1] = Storage<T>::encode(f.y);
  }
  *reinterpret_cast<V *>(p) = u.v;
}

// ---- Stochastic rounding ----
// Random bits from a counter-based hash: the 32-bit finaliser of Appleby's
// MurmurHash3 (a bijection of 32-bit words with full avalanche), applied to
// the step count, then the row, then (column, field).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Two FP32 values to one packed pair, each rounded up or down at random with
// the probability that makes its expected value exact (cvt.rs, sm_100
// family); `lo` lands in the low half (the lower address).
__device__ __forceinline__ uint32_t pack_sr(__half, float lo, float hi,
                                            uint32_t bits) {
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(bits));
  return d;
}
__device__ __forceinline__ uint32_t pack_sr(__nv_bfloat16, float lo, float hi,
                                            uint32_t bits) {
  uint32_t d;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(bits));
  return d;
}

// One output row (three fields) of a 16-bit format with stochastic
// rounding, kC / 2 column pairs each: one hashed word per column pair, from
// `key` (row and step) and the pair's first column x + 2q; the fields take
// that word rotated by 0, 11 and 22 bits.
template <int kC, typename T>
__device__ __forceinline__ void store_row_sr(T *dd, T *dx, T *dy,
                                             const float2 (&d)[kC / 2],
                                             const float2 (&jx)[kC / 2],
                                             const float2 (&jy)[kC / 2],
                                             uint32_t key, uint32_t x) {
  static_assert(kC % 2 == 0, "pairs of columns");
  const float2 sd = make_float2(Storage<T>::kD, Storage<T>::kD);
  const float2 sj = make_float2(Storage<T>::kJ, Storage<T>::kJ);
  uint32_t wd[kC / 2], wx[kC / 2], wy[kC / 2];
#pragma unroll
  for (int q = 0; q < kC / 2; ++q) {
    const uint32_t h = fmix32(key + (x + 2u * q) * 0x9e3779b1u);
    const float2 a = __fmul2_rn(d[q], sd), b = __fmul2_rn(jx[q], sj),
                 c = __fmul2_rn(jy[q], sj);
    wd[q] = pack_sr(T(), a.x, a.y, h);
    wx[q] = pack_sr(T(), b.x, b.y, __funnelshift_l(h, h, 11));
    wy[q] = pack_sr(T(), c.x, c.y, __funnelshift_l(h, h, 22));
  }
  if constexpr (kC == 4) {
    *reinterpret_cast<uint2 *>(dd) = make_uint2(wd[0], wd[1]);
    *reinterpret_cast<uint2 *>(dx) = make_uint2(wx[0], wx[1]);
    *reinterpret_cast<uint2 *>(dy) = make_uint2(wy[0], wy[1]);
  } else {
    *reinterpret_cast<uint32_t *>(dd) = wd[0];
    *reinterpret_cast<uint32_t *>(dx) = wx[0];
    *reinterpret_cast<uint32_t *>(dy) = wy[0];
  }
}

// FP32 storage with stochastic rounding: the dither, uniform in (-1/2, 1/2)
// and drawn once per step from the step count, in units of 2^-23 times the
// power of two that leads a stored value, i.e. of that value's unit in the
// last place.  Adding dither * lead(a) to an increment b before the rounded
// sum a + b makes the expected stored value exact (subtractive dither over
// one quantisation step); it is the same for every node of a step.
__device__ __forceinline__ float fp32_dither(uint32_t step) {
  const uint32_t h = fmix32(step * 0x9e3779b1u + 0x7f4a7c15u);
  const float r = (static_cast<float>(h >> 8) + 0.5f) * 0x1p-24f - 0.5f;
  return r * 0x1p-23f;
}

// The power of two at or below |a| for normal a (its exponent bits), else 0.
__device__ __forceinline__ float2 lead_pow2(float2 a) {
  return make_float2(__int_as_float(__float_as_int(a.x) & 0x7f800000),
                     __int_as_float(__float_as_int(a.y) & 0x7f800000));
}

// One source row as loaded, as column pairs (pair q: columns 2q, 2q + 1 of
// the lane's kC), with what the step derives from it once: z, the momentum
// the row's nodes contribute as sources (j, or -F at a solid node, whose
// equilibrium then has zero momentum j + F).
template <int kC>
struct RowP {
  float2 d[kC / 2], jx[kC / 2], jy[kC / 2];
  float2 zx[kC / 2], zy[kC / 2];
  unsigned solid;  // bit j: column j is solid or outside a non-periodic edge
  unsigned fluid;  // bit j: column j is a fluid node
};

// gathers bit 0 of each of the kC low bytes of v into bits 0..kC-1
template <int kC>
__device__ __forceinline__ unsigned byte_bits(unsigned v) {
  if constexpr (kC == 4) {
    v &= 0x01010101u;
    return (v | (v >> 7) | (v >> 14) | (v >> 21)) & 0xFu;
  } else {
    v &= 0x0101u;
    return (v | (v >> 7)) & 0x3u;
  }
}

// ---- Row staging through shared memory with the bulk-copy (TMA) engine ----
// Every warp tile streams its source rows through a ring of kS shared-memory
// stages: lane 0 starts `cp.async.bulk` global->shared copies of the tile's
// row window (three fields and the node types) several rows ahead, each
// completing on the stage's mbarrier, so the loads in flight do not occupy
// registers.  Every wait is bounded in time; on expiry the kernel raises
// kFlagCopyTimeout, drains its copies (again bounded) and stops.
constexpr unsigned kFlagUnstable = 1u;
constexpr unsigned kFlagCopyTimeout = 2u;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // one second

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// completes the current phase without data (a stage use that copies nothing)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src,
                                          uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0u;
}

// Waits for phase `parity` of `bar`; false when `limit` ns pass first.  A
// zero limit gives up at once, without looking.
__device__ __forceinline__ bool mbar_wait(
    uint64_t *bar, uint32_t parity,
    unsigned long long limit = kWaitLimitNs) {
  if (limit == 0ull) return false;
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Geometry of one ring stage for kC columns per lane: the field window starts
// at ws, the 16-byte boundary at or below the warp's first column x0 - kC,
// and covers its kLanes * kC columns; the node-type window starts at the
// 16-byte boundary at or below ws.  Two side slots after them hold, on a
// periodic x axis, 16-byte blocks (three fields, node types) from the other
// end of the row: the first the blocks that start the row (columns nx and
// nx + 1 seen from the domain's last column), the second (multiphase step)
// the blocks holding column nx - 2 (column -2 seen from the first).
template <int kC, typename T>
struct Stage {
  static constexpr int kAlignElems = 16 / static_cast<int>(sizeof(T));
  static constexpr int kWin =
      (kAlignElems - 1 + kLanes * kC + kAlignElems - 1) / kAlignElems * kAlignElems;
  static constexpr int kFieldBytes = kWin * static_cast<int>(sizeof(T));
  static constexpr int kMaskBytes = (kWin + 15 + 15) / 16 * 16;
  static constexpr int kSideBytes = 8 * 16;
  static constexpr int kBytes = 3 * kFieldBytes + kMaskBytes + kSideBytes;
};

// Sums of w_k (1, c_k) over the solid neighbours of a node, indexed by the
// 3 x 3 solid bits around it: bits 0-2 the row below (SW, S, SE), 3-5 its own
// row (W, -, E), 6-8 the row above (NW, N, NE).  c_k = -e_k points from the
// neighbour to the node.
struct alignas(16) SolidSums {
  float s0, sx, sy, pad;
};

__device__ __forceinline__ void build_solid_lut(SolidSums *lut) {
  for (int c = threadIdx.x; c < 512; c += blockDim.x) {
    const float sw = (c >> 0) & 1, s = (c >> 1) & 1, se = (c >> 2) & 1;
    const float w = (c >> 3) & 1, e = (c >> 5) & 1;
    const float nw = (c >> 6) & 1, n = (c >> 7) & 1, ne = (c >> 8) & 1;
    SolidSums v;
    v.s0 = k1_9 * ((w + e) + (s + n)) + k1_36 * ((sw + se) + (nw + ne));
    v.sx = k1_9 * (w - e) + k1_36 * ((sw - se) + (nw - ne));
    v.sy = k1_9 * (s - n) + k1_36 * ((sw + se) - (nw + ne));
    v.pad = 0.f;
    lut[c] = v;
  }
}

// Shared-memory footprint of one warp's ring and of a block.
template <typename T, int kC, int kS>
__host__ __device__ constexpr int ring_bytes() {
  return 128 + kS * Stage<kC, T>::kBytes;  // barriers, then the stages
}

template <typename T, int kC, int kS>
__host__ __device__ constexpr int smem_bytes() {
  return 512 * static_cast<int>(sizeof(SolidSums)) +
         kWarps * ring_bytes<T, kC, kS>();
}

// The batched kernel's block adds one launch-state slot per warp after the
// rings.
template <typename T, int kC, int kS>
__host__ __device__ constexpr int batch_smem_bytes() {
  return smem_bytes<T, kC, kS>() +
         kWarps * ((static_cast<int>(sizeof(StepLaunch)) + 15) / 16 * 16);
}

// The step kernel's warp tile.  kC columns per lane (4: 16-byte rows of
// FP32, 2: 8-byte rows), kRows output rows per warp (even).  The warp marches
// down its tile one source row s at a time; all per-node arithmetic runs on
// column pairs of that row with the packed FP32 instructions.  Row s adds
//   North(s) to output row s - 1, Same(s) to row s, South(s) to row s + 1,
// so output row s - 1 completes when row s arrives:
//   out(s - 1) = South(s - 2) + Same(s - 1) + North(s),
// and the warp carries acc = South(s - 2) + Same(s - 1) and South(s - 1)
// from one row to the next, with the raw row s - 1 (the old values of the
// nodes it completes).  Clean tiles (and the multiphase step) take rows two
// per loop turn with the roles of the two row buffers swapped, so carrying
// them costs no register moves; the general code takes one row per turn and
// copies it into the previous-row buffer, which halves its loop's code.
//
// warp w (0 .. kWarps - 1, stacked in y) of block tile (bx, by) covers
// (30 kC) columns x kRows rows.  `gx` is the number of block tiles along x
// (for the index of the warp's reduction partial); `slot` is the calling
// warp's place in its block, which owns a shared-memory ring.  Every lane of
// the warp calls it; no other warp takes part.  kClean: the warp tile's
// marched rows and columns all lie inside the domain and hold fluid nodes
// only (see tile_flags_kernel), so node types, edges and wall terms need no
// handling and the node-type rows are not copied.  kSC: the Shan-Chen
// multiphase step (Section 4, Eq. f_sc), see the force pipeline below.
template <typename T, int kC, int kRows, int kS, bool kReduce, bool kClean,
          bool kSC = false>
__device__ __forceinline__ void step_tile(const StepLaunch &a, int64_t bx,
                                          int64_t by, int w, int slot,
                                          int64_t gx, const SolidSums *lut,
                                          unsigned char *smem) {
  static_assert(kRows % 2 == 0, "rows per warp must be even");
  static_assert(kS >= 4 && kS % 2 == 0 && kS <= 16, "ring stages");
  static_assert(kC == 2 || kC == 4, "columns per lane");
  constexpr int kP = kC / 2;  // column pairs per lane
  constexpr int kTile = (kLanes - 2) * kC;
  constexpr bool kF32 = std::is_same<T, float>::value;
  using St = Stage<kC, T>;
  using SS = Storage<T>;
  using Row = RowP<kC>;

  const int lane = threadIdx.x & (kLanes - 1);
  const int64_t x0 = bx * kTile;
  const int64_t xb = x0 - kC + static_cast<int64_t>(kC) * lane;
  const int64_t y0 = (by * kWarps + w) * kRows;
  const int64_t y1 = min(y0 + kRows, a.ny);
  const bool owner = lane >= 1 && lane <= kLanes - 2 && xb < a.nx;
  // columns of this lane that are outputs inside the domain (reductions)
  unsigned out_cols = 0u;
#pragma unroll
  for (int j = 0; j < kC; ++j) out_cols |= (owner && xb + j < a.nx) << j;
  // Row windows.  Of the field window [ws, ws + kWin) and the node-type
  // window [m0, m0 + kMaskBytes), the bulk copies fill the part inside the
  // row, [c0, c1) and [k0, k1), rounded out to 16-byte boundaries (which stay
  // inside the row's pitch).  Other columns read as solid, except that on a
  // periodic x axis column -1 is column nx - 1 and column nx is column 0: the
  // 16-byte blocks holding those land in the window head (the tile at x = 0
  // starts its window one block left of the domain) and in the side slot.
  const int64_t ws = (x0 - kC) & ~int64_t(St::kAlignElems - 1);
  const int64_t m0 = ws & ~int64_t(15);
  const bool interior = ws >= 0 && ws + St::kMaskBytes <= a.nx;
  const bool wrap_l = a.periodic_x && ws < 0;
  const bool wrap_r = a.periodic_x && a.nx < x0 + (kLanes - 1) * kC;
  // this lane's columns that lie in the domain, and the one (if any) that is
  // column -1 or nx of a periodic x axis, read from the wrapped blocks
  unsigned in_cols = 0u;
#pragma unroll
  for (int j = 0; j < kC; ++j)
    in_cols |= (xb + j >= 0 && xb + j < a.nx) << j;
  int wrap_col = -1;
  if (wrap_l && xb < 0) wrap_col = kC - 1;            // column -1
  if (wrap_r && xb <= a.nx && a.nx < xb + kC)          // column nx
    wrap_col = static_cast<int>(a.nx - xb);
  unsigned char *ring =
      smem + 512 * sizeof(SolidSums) + slot * ring_bytes<T, kC, kS>();
  uint64_t *bars = reinterpret_cast<uint64_t *>(ring);
  unsigned char *stages = ring + 128;
  const int c_lane = static_cast<int>(x0 - kC - ws) + kC * lane;
  const int m_lane = static_cast<int>(ws - m0) + c_lane;
  const float fx = a.fx, fy = a.fy;
  const float2 F2x = bc(fx), F2y = bc(fy), F22y = bc(2.0f * fy);
  const float2 one = bc(1.0f), c3 = bc(3.0f), cm15 = bc(-1.5f);
  const float2 w1_9 = bc(k1_9), w1_36 = bc(k1_36), w1_12 = bc(k1_12),
               w1_3 = bc(k1_3), w4_9 = bc(k4_9), w1_6 = bc(k1_6),
               wm1_6 = bc(-k1_6), half = bc(0.5f), quarter = bc(0.25f);
  // FP32 storage with stochastic rounding: this step's dither
  const float2 dither = bc(kF32 && a.sr ? fp32_dither(a.step) : 0.0f);

  // Residual sums in FP32 per lane (at most 64 rows x 4 columns of a tile),
  // FP64 from the warp sums on: non-negative terms, a lane's rounding error a
  // few 1e-6 of its own sum.  The mass is a compensated (Kahan) FP32 sum of
  // the lane's row sums: deviations of order one (a multiphase vapour) keep
  // it to about 1e-7 of a lane's sum.
  float2 rs_num = bc(0.f), rs_den = bc(0.f);
  float rs_mass = 0.f, rs_comp = 0.f;
  float rmin = 1.0f;

  if (y0 < a.ny) {
    // Row indices in 32 bits: the launchers reject ny >= 2^30.
    const int ty0 = static_cast<int>(y0), ty1 = static_cast<int>(y1);
    const int tny = static_cast<int>(a.ny);
    const int npairs = (ty1 - ty0 + 1) / 2 + 1;
    // Ring rows: the source rows y0 - 1 .. y0 - 2 + 2 npairs and, for the
    // multiphase step, one more row above and below them whose potential the
    // force of the outermost source rows needs (kLead: rows before the
    // first source row).
    constexpr int kLead = kSC ? 1 : 0;
    const int nrows = 2 * npairs + 2 * kLead;
    // grid row of ring index i: -1 for a solid row beyond a wall-less edge
    auto source_row = [&](int i) -> int {
      const int r = ty0 - 1 - kLead + i;
      if (r >= 0 && r < tny) return r;
      return a.periodic_y ? static_cast<int>(wrap_index(r, tny)) : -1;
    };
    // starts the copies of ring row i into stage st (lane 0 only)
    auto issue = [&](int i, int st) {
      // a clean tile's rows all lie inside the domain
      const int r = kClean ? ty0 - 1 - kLead + i : source_row(i);
      uint64_t *bar = bars + st;
      if (r < 0) {  // solid row: nothing to copy, but the phase still completes
        mbar_arrive(bar);
        return;
      }
      unsigned char *dst = stages + st * St::kBytes;
      unsigned char *dmask = dst + 3 * St::kFieldBytes;
      // the whole window lies in the row, or (clean tile) at most 16 bytes
      // past its last column, which the lanes do not read
      if (kClean || interior) {
        const int64_t off = static_cast<int64_t>(r) * a.pitch + ws;
        mbar_expect_tx(bar, 3 * St::kFieldBytes + (kClean ? 0 : St::kMaskBytes));
        bulk_copy(dst, static_cast<const T *>(a.src.d) + off, St::kFieldBytes,
                  bar);
        bulk_copy(dst + St::kFieldBytes,
                  static_cast<const T *>(a.src.jx) + off, St::kFieldBytes, bar);
        bulk_copy(dst + 2 * St::kFieldBytes,
                  static_cast<const T *>(a.src.jy) + off, St::kFieldBytes, bar);
        if (!kClean)
          bulk_copy(dmask, a.mask + r * a.pitch + m0, St::kMaskBytes, bar);
        return;
      }
      constexpr int64_t kA = St::kAlignElems;
      const int64_t c0 = max(ws, int64_t(0));
      const int64_t c1 = min(ws + St::kWin, (a.nx + kA - 1) & ~(kA - 1));
      const int64_t k0 = max(m0, int64_t(0));
      const int64_t k1 = min(m0 + St::kMaskBytes, (a.nx + 15) & ~int64_t(15));
      const uint32_t fbytes = static_cast<uint32_t>((c1 - c0) * sizeof(T));
      const uint32_t mbytes = kClean ? 0u : static_cast<uint32_t>(k1 - k0);
      mbar_expect_tx(bar, 3 * fbytes + mbytes + (wrap_l ? 64u : 0u) +
                              (wrap_r ? 64u : 0u) +
                              (kSC && wrap_l ? 64u : 0u));
      const int64_t rp = static_cast<int64_t>(r) * a.pitch;
      const T *src[3] = {static_cast<const T *>(a.src.d) + rp,
                         static_cast<const T *>(a.src.jx) + rp,
                         static_cast<const T *>(a.src.jy) + rp};
      const uint8_t *mrow = a.mask + rp;
      const int64_t foff = (c0 - ws) * static_cast<int64_t>(sizeof(T));
#pragma unroll
      for (int f = 0; f < 3; ++f)
        bulk_copy(dst + f * St::kFieldBytes + foff, src[f] + c0, fbytes, bar);
      if (!kClean) bulk_copy(dmask + (k0 - m0), mrow + k0, mbytes, bar);
      if (wrap_l) {  // the blocks holding column nx - 1, into the window head
        const int64_t lf = (a.nx - 1) & ~(kA - 1), lm = (a.nx - 1) & ~int64_t(15);
#pragma unroll
        for (int f = 0; f < 3; ++f)
          bulk_copy(dst + f * St::kFieldBytes, src[f] + lf, 16u, bar);
        bulk_copy(dmask, mrow + lm, 16u, bar);
      }
      if (wrap_r) {  // the blocks holding column 0, into the side slot
        unsigned char *side = dmask + St::kMaskBytes;
#pragma unroll
        for (int f = 0; f < 3; ++f) bulk_copy(side + 16 * f, src[f], 16u, bar);
        bulk_copy(side + 48, mrow, 16u, bar);
      }
      if (kSC && wrap_l) {  // the blocks holding column -2, second side slot
        unsigned char *side2 = dmask + St::kMaskBytes + 64;
        const int64_t l2 = a.nx >= 2 ? a.nx - 2 : 0;
#pragma unroll
        for (int f = 0; f < 3; ++f)
          bulk_copy(side2 + 16 * f, src[f] + (l2 & ~(kA - 1)), 16u, bar);
        bulk_copy(side2 + 48, mrow + (l2 & ~int64_t(15)), 16u, bar);
      }
    };
    // value v into column `col` (0 .. kC - 1) of a row of pairs
    auto set_col = [](float2 (&p)[kP], int col, float v) {
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        if (col == 2 * q) p[q].x = v;
        if (col == 2 * q + 1) p[q].y = v;
      }
    };
    // ring row i, in stage st with phase parity ph -> registers; false when
    // the copy did not arrive in time
    auto fetch = [&](int i, int st, unsigned ph, Row &o) -> bool {
      if constexpr (kClean) {  // an in-domain row of fluid nodes
        const bool ok = mbar_wait(bars + st, ph, a.wait_ns);
        const unsigned char *src = stages + st * St::kBytes;
        load_pairs<kC, T>(reinterpret_cast<const T *>(src) + c_lane, o.d,
                          1.0f / SS::kD);
        load_pairs<kC, T>(
            reinterpret_cast<const T *>(src + St::kFieldBytes) + c_lane, o.jx,
            1.0f / SS::kJ);
        load_pairs<kC, T>(
            reinterpret_cast<const T *>(src + 2 * St::kFieldBytes) + c_lane,
            o.jy, 1.0f / SS::kJ);
        o.solid = 0u;
        o.fluid = (1u << kC) - 1u;
        return ok;
      }
      if (source_row(i) < 0) {
#pragma unroll
        for (int q = 0; q < kP; ++q) o.d[q] = o.jx[q] = o.jy[q] = bc(0.f);
        o.solid = (1u << kC) - 1u;
        o.fluid = 0u;
        return true;
      }
      const bool ok = mbar_wait(bars + st, ph, a.wait_ns);
      const unsigned char *src = stages + st * St::kBytes;
      const T *fd = reinterpret_cast<const T *>(src);
      const T *fx_ = reinterpret_cast<const T *>(src + St::kFieldBytes);
      const T *fy_ = reinterpret_cast<const T *>(src + 2 * St::kFieldBytes);
      const unsigned char *mw = src + 3 * St::kFieldBytes;
      load_pairs<kC, T>(fd + c_lane, o.d, 1.0f / SS::kD);
      load_pairs<kC, T>(fx_ + c_lane, o.jx, 1.0f / SS::kJ);
      load_pairs<kC, T>(fy_ + c_lane, o.jy, 1.0f / SS::kJ);
      const unsigned char *mk = mw + m_lane;
      unsigned m;
      if constexpr (kC == 4)
        m = *reinterpret_cast<const unsigned *>(mk);
      else
        m = *reinterpret_cast<const unsigned short *>(mk);
      // columns outside the domain are solid (whatever the window holds)
      o.solid = byte_bits<kC>(m) | (~in_cols & ((1u << kC) - 1u));
      o.fluid = byte_bits<kC>(~(m | (m >> 1))) & in_cols;
      if (wrap_col >= 0) {  // column -1 or nx of a periodic x axis
        const bool left = wrap_col == kC - 1 && xb < 0;
        // column nx - 1 in the window head, or column 0 in the side slot
        const int fo = static_cast<int>((a.nx - 1) & (St::kAlignElems - 1));
        const T *side = reinterpret_cast<const T *>(mw + St::kMaskBytes);
        set_col(o.d, wrap_col,
                SS::decode(left ? fd[fo] : side[0]) * (1.0f / SS::kD));
        set_col(o.jx, wrap_col,
                SS::decode(left ? fx_[fo] : side[St::kAlignElems]) *
                    (1.0f / SS::kJ));
        set_col(o.jy, wrap_col,
                SS::decode(left ? fy_[fo] : side[2 * St::kAlignElems]) *
                    (1.0f / SS::kJ));
        const unsigned t =
            left ? mw[(a.nx - 1) & 15] : mw[St::kMaskBytes + 48];
        const unsigned bit = 1u << wrap_col;
        o.solid = (o.solid & ~bit) | ((t == 1u) ? bit : 0u);
        o.fluid = (o.fluid & ~bit) | ((t == 0u) ? bit : 0u);
      }
      if constexpr (kSC) {
        // The multiphase force of columns -1 and nx needs the potential of
        // columns -2 and nx + 1 on a periodic x axis: their density and node
        // type (nothing else of theirs reaches an output) from the second
        // side slot and the first.
        auto patch = [&](int col, float d, unsigned t) {
          set_col(o.d, col, d);
          const unsigned bit = 1u << col;
          o.solid = (o.solid & ~bit) | ((t == 1u) ? bit : 0u);
          o.fluid = (o.fluid & ~bit) | ((t == 0u) ? bit : 0u);
        };
        const unsigned char *side = mw + St::kMaskBytes;
        if (wrap_l && xb < 0) {  // column -2: column nx - 2 (0 for nx < 2)
          const int64_t l2 = a.nx >= 2 ? a.nx - 2 : 0;
          const T *f2 = reinterpret_cast<const T *>(side + 64);
          patch(kC - 2,
                SS::decode(f2[l2 & (St::kAlignElems - 1)]) * (1.0f / SS::kD),
                side[64 + 48 + (l2 & 15)]);
        }
        if (wrap_r && xb <= a.nx + 1 && a.nx + 1 < xb + kC) {
          // column nx + 1: column 1 (0 for nx < 2), in the first side slot
          const int r2 = a.nx >= 2 ? 1 : 0;
          const T *f1 = reinterpret_cast<const T *>(side);
          patch(static_cast<int>(a.nx + 1 - xb),
                SS::decode(f1[r2]) * (1.0f / SS::kD), side[48 + r2]);
        }
      }
      return ok;
    };

    // Carried from row to row (see above): acc = South(s - 2) + Same(s - 1)
    // plus the vertical momentum difference with row s - 2, and South(s - 1).
    float2 acc_dd[kP], acc_mx[kP], acc_my[kP], t_dd[kP], t_mx[kP], t_my[kP];
    Row ra, rb;
#pragma unroll
    for (int q = 0; q < kP; ++q) {
      acc_dd[q] = acc_mx[q] = acc_my[q] = bc(0.f);
      t_dd[q] = t_mx[q] = t_my[q] = bc(0.f);
      rb.d[q] = rb.jx[q] = rb.jy[q] = rb.zx[q] = rb.zy[q] = bc(0.f);
    }
    rb.solid = rb.fluid = 0u;
    unsigned pS6 = 0u, ppS6 = 0u;  // solid bits (cols -1..kC) of rows s-1, s-2

    // The multiphase force (kSC), F_SC(x) = -g psi(x) sum_i w_i psi(x + e_i)
    // e_i (Eq. f_sc with Shan and Chen's psi = 1 - exp(-rho), alpha_i = w_i,
    // G(e_i) = -g e_i; psi = 0 at solid nodes and outside non-periodic
    // edges), needs the potentials of the rows above and below a source row.
    // The ring holds one row more above and below the source rows; when
    // source row s is taken, row s + 1 is read from its stage as well (it
    // stays there until taken in turn) and its potential terms computed
    // once.  With A = right - left and S = right + left of a row's
    // potentials and C the potentials themselves,
    //   F_SC(s) = -g C(s) (A(s)/9 + (A(s-1) + A(s+1))/36,
    //                      (C(s+1) - C(s-1))/9 + (S(s+1) - S(s-1))/36):
    // the rows above and below are combined first, so the force is exactly
    // odd under either mirror of the lattice, in floating point too, and a
    // symmetric drop feels no net force.  The terms of rows s - 1 and s are
    // carried, in two sets that swap roles each row as the row buffers do.
    const float2 mg = bc(-a.g_sc);
    // potential of a row's columns (C) and its horizontal differences and
    // sums (A = right - left, S = right + left)
    auto psi_terms = [&](const Row &r, float2 (&C)[kP], float2 (&A)[kP],
                         float2 (&S)[kP]) {
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        const float2 rho = add(r.d[q], one);
        const float2 e = make_float2(__expf(-rho.x), __expf(-rho.y));
        const bool s0 = (r.solid >> (2 * q)) & 1u;
        const bool s1 = (r.solid >> (2 * q + 1)) & 1u;
        C[q] = make_float2(s0 ? 0.f : 1.0f - e.x, s1 ? 0.f : 1.0f - e.y);
      }
      const float hm = __shfl_up_sync(kFull, C[kP - 1].y, 1);
      const float hp = __shfl_down_sync(kFull, C[0].x, 1);
      // column by column, as for the row's other neighbour terms
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        const float l0 = q == 0 ? hm : C[q - 1].y, l1 = C[q].x;
        const float r0 = C[q].y, r1 = q == kP - 1 ? hp : C[q + 1].x;
        A[q] = make_float2(__fsub_rn(r0, l0), __fsub_rn(r1, l1));
        S[q] = make_float2(__fadd_rn(r0, l0), __fadd_rn(r1, l1));
      }
    };
    // Source row s = ty0 - 1 + i, fetched into `cur`; `prev` holds row s - 1.
    // kSC: `nxt` holds row s + 1 (its density and node types are used),
    // (pC, pA, pS) the potential terms of row s - 1, (cC, cA, cS) those of
    // row s; row s + 1's replace row s - 1's.
    auto row = [&](int i, Row &cur, const Row &prev, const Row &nxt,
                   float2 (&pC)[kP], float2 (&pA)[kP], float2 (&pS)[kP],
                   float2 (&cC)[kP], float2 (&cA)[kP], float2 (&cS)[kP]) {
      const int s = ty0 - 1 + i;
      float2 Fsx[kP], Fsy[kP];  // F_SC of row s
      if constexpr (kSC) {
        float2 C1[kP], A1[kP], S1[kP];
        psi_terms(nxt, C1, A1, S1);
#pragma unroll
        for (int q = 0; q < kP; ++q) {
          const float2 k = mul(cC[q], mg);
          const float2 sx = fma2(w1_36, add(pA[q], A1[q]), mul(w1_9, cA[q]));
          const float2 sy =
              fma2(w1_9, sub(C1[q], pC[q]), mul(w1_36, sub(S1[q], pS[q])));
          Fsx[q] = mul(k, sx);
          Fsy[q] = mul(k, sy);
          pC[q] = C1[q];
          pA[q] = A1[q];
          pS[q] = S1[q];
        }
      }
      const int o = s - 1;                       // output row completed here
      const bool out_row = o >= ty0 && o < ty1;  // the same for the warp
      // Per-node quantities of row s, pre-scaled by the lattice weights they
      // meet (K = (delta + A) / 9, G / 36, X / 36 with A = 3 Pxx - 1.5 Pyy,
      // G = delta + 3 tr Pi, X = 9 Pxy), so that each neighbour combination
      // below is a sum or a difference.
      float2 K[kP], G[kP], X[kP], P[kP], R0[kP];
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        float2 dfj;
        // z: the momentum a node brings as a source, its own j plus (kSC)
        // its multiphase force; a solid node brings -F (zero momentum j + F)
        const float2 jx = kSC ? add(cur.jx[q], Fsx[q]) : cur.jx[q];
        const float2 jy = kSC ? add(cur.jy[q], Fsy[q]) : cur.jy[q];
        if constexpr (kClean) {
          cur.zx[q] = jx;
          cur.zy[q] = jy;
          dfj = cur.d[q];
        } else {
          const bool s0 = (cur.solid >> (2 * q)) & 1u;
          const bool s1 = (cur.solid >> (2 * q + 1)) & 1u;
          cur.zx[q] = make_float2(s0 ? -fx : jx.x, s1 ? -fx : jx.y);
          cur.zy[q] = make_float2(s0 ? -fy : jy.x, s1 ? -fy : jy.y);
          dfj = make_float2(s0 ? 0.f : cur.d[q].x, s1 ? 0.f : cur.d[q].y);
        }
        const float2 mx = add(cur.zx[q], F2x);  // j + F, 0 on solid nodes
        const float2 my = add(cur.zy[q], F2y);
        const float2 rho = add(dfj, one);
        const float2 ir =
            make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
        const float2 t = mul(mx, ir);
        const float2 pxx = mul(t, mx), pxy = mul(t, my);
        const float2 pyy = mul(mul(my, my), ir);
        const float2 tr = add(pxx, pyy);
        K[q] = fma2(w1_9, dfj, fma2(w1_3, pxx, mul(wm1_6, pyy)));
        P[q] = fma2(c3, pyy, fma2(cm15, pxx, dfj));  // delta + 3 Pyy - 1.5 Pxx
        G[q] = fma2(w1_12, tr, mul(w1_36, dfj));
        X[q] = mul(quarter, pxy);
        R0[q] = fma2(cm15, tr, dfj);
      }
      // Left and right neighbours: the columns -1 and kC of a row come from
      // the neighbouring lanes; the sums and differences of a pair's left
      // and right neighbours are formed column by column (scalar adds round
      // as the packed ones do, and need no register moves to pair up
      // neighbouring columns).
      struct Halo {
        float m, p;
      };
      auto halo = [&](const float2 (&v)[kP]) -> Halo {
        return {__shfl_up_sync(kFull, v[kP - 1].y, 1),
                __shfl_down_sync(kFull, v[0].x, 1)};
      };
      const Halo hK = halo(K), hG = halo(G), hX = halo(X);
      const Halo hZx = halo(cur.zx), hZy = halo(cur.zy);
      unsigned S6 = 0u;
      bool any_solid = false;
      if constexpr (!kClean) {
        const unsigned sl = __shfl_up_sync(kFull, cur.solid, 1);
        const unsigned sr = __shfl_down_sync(kFull, cur.solid, 1);
        S6 = ((sl >> (kC - 1)) & 1u) | (cur.solid << 1) |
             ((sr & 1u) << (kC + 1));
        any_solid = __any_sync(kFull, (ppS6 | pS6 | S6) != 0u);
      }

      float2 od[kP], ox[kP], oy[kP];
      float mrow = 0.f;  // this row's mass terms (kReduce)
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        const float2 zxC = cur.zx[q], zyC = cur.zy[q];
        // column j (-1 .. kC) of a row of pairs with its halo columns
        auto col = [](const float2 (&v)[kP], const Halo &h, int j) -> float {
          return j < 0 ? h.m : j >= kC ? h.p
                                       : ((j & 1) ? v[j >> 1].y : v[j >> 1].x);
        };
        // the pair's left neighbours are columns 2q - 1, 2q and its right
        // ones 2q + 1, 2q + 2: left + right, left - right, and the
        // differences of a side with the pair itself
        auto lpr = [&](const float2 (&v)[kP], const Halo &h) {
          return make_float2(__fadd_rn(col(v, h, 2 * q - 1), col(v, h, 2 * q + 1)),
                             __fadd_rn(col(v, h, 2 * q), col(v, h, 2 * q + 2)));
        };
        auto lmr = [&](const float2 (&v)[kP], const Halo &h) {
          return make_float2(__fsub_rn(col(v, h, 2 * q - 1), col(v, h, 2 * q + 1)),
                             __fsub_rn(col(v, h, 2 * q), col(v, h, 2 * q + 2)));
        };
        auto side = [&](const float2 (&v)[kP], const Halo &h, int j0,
                        float2 c) {
          return make_float2(__fsub_rn(col(v, h, j0), c.x),
                             __fsub_rn(col(v, h, j0 + 1), c.y));
        };
        const float2 Ks = lpr(K, hK), Kd = lmr(K, hK);
        const float2 Gs = lpr(G, hG), Gd = lmr(G, hG);
        const float2 Xs = lpr(X, hX), Xd = lmr(X, hX);
        const float2 mxd = lmr(cur.zx, hZx), myd = lmr(cur.zy, hZy);
        const float2 mys = add(lpr(cur.zy, hZy), F22y);
        const float2 hx = add(side(cur.zx, hZx, 2 * q - 1, zxC),  // exact
                              side(cur.zx, hZx, 2 * q + 1, zxC));
        const float2 hy = add(side(cur.zy, hZy, 2 * q - 1, zyC),
                              side(cur.zy, hZy, 2 * q + 1, zyC));
        // Row s as the row above output row s - 1 (N: NW, N, NE) and below
        // output row s + 1 (T: SW, S, SE).  The two share their terms up to
        // signs:
        //   U = P/9 + Gs + mxd/12,  V = (zy_C + Fy)/3 + Xd + mys/12,
        //   Y = Xd + hy/12,  U' = Gd + hx/12,  V' = Xs + myd/12,
        //   N = (U - V, U' - V', Y - U),  T = (U + V, U' + V', Y + U)
        // for (delta, jx, jy).
        const float2 U = fma2(w1_9, P[q], fma2(w1_12, mxd, Gs));
        const float2 V = fma2(w1_3, add(zyC, F2y), fma2(w1_12, mys, Xd));
        const float2 Y = fma2(w1_12, hy, Xd);
        const float2 Up = fma2(w1_12, hx, Gd), Vp = fma2(w1_12, myd, Xs);
        // Row s as the own row of output row s (W, O, E)
        const float2 Sdd = fma2(w4_9, R0[q], fma2(w1_3, mxd, Ks));
        const float2 Smx = fma2(w1_3, hx, Kd);

        // Output row s - 1: the momentum in increment form on the base z_O
        // (j_O, plus F_SC(O) for the multiphase step), every z_P - z_O an
        // exact difference; solid neighbours add their wall terms in place
        // (nothing to add, and no zero terms, without solids).
        const float2 dO = prev.d[q], jxO = prev.jx[q], jyO = prev.jy[q];
        const float2 zxO = prev.zx[q], zyO = prev.zy[q];
        float2 dn = add(acc_dd[q], sub(U, V));
        float2 incx = fma2(w1_6, sub(zxC, zxO),
                           add(add(acc_mx[q], sub(Up, Vp)), F2x));
        float2 incy = fma2(half, sub(zyC, zyO),
                           add(add(acc_my[q], sub(Y, U)), F2y));
        if (!kClean && any_solid) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int j = 2 * q + e;
            const unsigned c = ((ppS6 >> j) & 7u) | (((pS6 >> j) & 7u) << 3) |
                               (((S6 >> j) & 7u) << 6);
            const SolidSums E = lut[c];
            if (e == 0) {
              dn.x = fmaf(dO.x, E.s0, dn.x);
              incx.x = fmaf(dO.x, E.sx, incx.x);
              incy.x = fmaf(dO.x, E.sy, incy.x);
            } else {
              dn.y = fmaf(dO.y, E.s0, dn.y);
              incx.y = fmaf(dO.y, E.sx, incx.y);
              incy.y = fmaf(dO.y, E.sy, incy.y);
            }
          }
        }
        if constexpr (kF32) {
          if (a.sr) {  // stochastic rounding of the stored momentum
            incx = fma2(lead_pow2(zxO), dither, incx);
            incy = fma2(lead_pow2(zyO), dither, incy);
          }
        }
        const float2 mxn = add(zxO, incx);
        const float2 myn = add(zyO, incy);
        bool f0 = true, f1 = true;
        if constexpr (!kClean) {
          f0 = (prev.fluid >> (2 * q)) & 1u;
          f1 = (prev.fluid >> (2 * q + 1)) & 1u;
          od[q] = make_float2(f0 ? dn.x : dO.x, f1 ? dn.y : dO.y);
          ox[q] = make_float2(f0 ? mxn.x : jxO.x, f1 ? mxn.y : jxO.y);
          oy[q] = make_float2(f0 ? myn.x : jyO.x, f1 ? myn.y : jyO.y);
        } else {
          od[q] = dn;
          ox[q] = mxn;
          oy[q] = myn;
        }
        if constexpr (kReduce && !kClean) {
          // The residual's terms.  u_new - u_old = ((j_n - j_o) -
          // u_o (d_n - d_o)) / rho_n: the step's own changes, no cancellation
          // between two O(|u|) values; u_o is taken as j_o / rho_n, which
          // errs by the relative density change of the step in this
          // second-order term only.  So (|u_n - u_o|^2, |u_n|^2) =
          // (|e|^2, |j_n|^2) / rho_n^2 with e = (j_n - j_o) -
          // j_o (d_n - d_o) / rho_n, the division by rho_n^2 folded into the
          // accumulating FMAs.  Only valid nodes add (fluid, owned, in an
          // output row).
          const float2 rn = add(dn, one);
          const float2 irn =
              make_float2(__fdividef(1.0f, rn.x), __fdividef(1.0f, rn.y));
          const float2 irn2 = mul(irn, irn);
          const float2 t = mul(sub(dO, dn), irn);
          const float2 ex = fma2(jxO, t, sub(mxn, jxO));
          const float2 ey = fma2(jyO, t, sub(myn, jyO));
          const float2 nn = fma2(ex, ex, mul(ey, ey));
          const float2 dd2 = fma2(mxn, mxn, mul(myn, myn));
          const bool v0 = f0 && out_row && ((out_cols >> (2 * q)) & 1u);
          const bool v1 = f1 && out_row && ((out_cols >> (2 * q + 1)) & 1u);
          if (v0) {
            rs_num.x = fmaf(nn.x, irn2.x, rs_num.x);
            rs_den.x = fmaf(dd2.x, irn2.x, rs_den.x);
            mrow += dn.x;
            rmin = fminf(rmin, rn.x);
          }
          if (v1) {
            rs_num.y = fmaf(nn.y, irn2.y, rs_num.y);
            rs_den.y = fmaf(dd2.y, irn2.y, rs_den.y);
            mrow += dn.y;
            rmin = fminf(rmin, rn.y);
          }
        }
        // carry to output row s: South(s - 1) + Same(s) and the vertical
        // difference with row s - 1 (j of row s is the base of its nodes)
        acc_dd[q] = add(t_dd[q], Sdd);
        acc_mx[q] = fma2(w1_6, sub(prev.zx[q], cur.zx[q]), add(t_mx[q], Smx));
        acc_my[q] = fma2(half, sub(prev.zy[q], cur.zy[q]), t_my[q]);
        t_dd[q] = add(U, V);
        t_mx[q] = add(Up, Vp);
        t_my[q] = add(Y, U);
      }
      if constexpr (kReduce && kClean) {
        // The same terms as the general code's, in the same order; every
        // lane sums its row (the halo lanes' sums are dropped at the end of
        // the tile), as one block after the row's arithmetic.
        if (out_row) {
#pragma unroll
          for (int q = 0; q < kP; ++q) {
            const float2 dn = od[q], mxn = ox[q], myn = oy[q];
            const float2 dO = prev.d[q], jxO = prev.jx[q], jyO = prev.jy[q];
            const float2 rn = add(dn, one);
            const float2 irn =
                make_float2(__fdividef(1.0f, rn.x), __fdividef(1.0f, rn.y));
            const float2 irn2 = mul(irn, irn);
            const float2 t = mul(sub(dO, dn), irn);
            const float2 ex = fma2(jxO, t, sub(mxn, jxO));
            const float2 ey = fma2(jyO, t, sub(myn, jyO));
            const float2 nn = fma2(ex, ex, mul(ey, ey));
            const float2 dd2 = fma2(mxn, mxn, mul(myn, myn));
            rs_num = fma2(nn, irn2, rs_num);
            rs_den = fma2(dd2, irn2, rs_den);
            mrow += dn.x;
            mrow += dn.y;
            rmin = fminf(rmin, fminf(rn.x, rn.y));
          }
        }
      }
      if constexpr (kReduce) {
        if (out_row) {  // compensated sum of the rows (uniform branch)
          const float y = __fsub_rn(mrow, rs_comp);
          const float t = __fadd_rn(rs_mass, y);
          rs_comp = __fsub_rn(__fsub_rn(t, rs_mass), y);
          rs_mass = t;
        }
      }
      if (owner && out_row) {
        T *dd = static_cast<T *>(a.dst.d);
        T *dx = static_cast<T *>(a.dst.jx);
        T *dy = static_cast<T *>(a.dst.jy);
        const int64_t off = static_cast<int64_t>(o) * a.pitch + xb;
        bool stored = false;
        if constexpr (!kF32) {
          if (a.sr) {  // uniform across the warp
            stored = true;
            const uint32_t xs = static_cast<uint32_t>(xb);
            // one key per (row, step)
            const uint32_t key =
                fmix32(fmix32(a.step) ^ (static_cast<uint32_t>(o) * 0x85ebca77u));
            store_row_sr<kC, T>(dd + off, dx + off, dy + off, od, ox, oy, key,
                                xs);
          }
        }
        if (!stored) {
          store_pairs<kC, T>(dd + off, od, SS::kD);
          store_pairs<kC, T>(dx + off, ox, SS::kJ);
          store_pairs<kC, T>(dy + off, oy, SS::kJ);
        }
      }
      ppS6 = pS6;
      pS6 = S6;
    };

    // Ring rows are taken in order, so the stage and phase parity of the
    // next row to take (tst, tph) and the stage of the next row to issue
    // (ist) advance by one per row instead of being divided out.
    int issued = 0, ist = 0, tst = 0;
    unsigned tph = 0u;
    if (lane == 0) {
      for (int st = 0; st < kS; ++st) mbar_init(bars + st);
      fence_async_shared();
      for (; issued < nrows && issued < kS; ++issued) issue(issued, issued);
    }
    issued = __shfl_sync(kFull, issued, 0);
    ist = issued == kS ? 0 : issued;
    __syncwarp();
    // takes ring row i into `r` and refills its stage; false on a timeout
    // releases the stage of the row just read: refills it with the next ring
    // row to issue, and advances to the next row to take
    auto release = [&]() {
      __syncwarp();  // every lane has read the stage
      if (issued < nrows) {
        if (lane == 0) {
          fence_async_shared();
          issue(issued, ist);
        }
        ++issued;
        ist = ist + 1 == kS ? 0 : ist + 1;
      }
      if (++tst == kS) {
        tst = 0;
        tph ^= 1u;
      }
    };
    auto take = [&](int i, Row &r) -> bool {
      const bool ok = fetch(i, tst, tph, r);
      if (!__all_sync(kFull, ok)) return false;
      release();
      return true;
    };
    // kSC: takes ring row i, which `peeked` was just read from by peek: its
    // values are in registers already, so only the stage is released
    auto take_peeked = [&](int i, Row &r, const Row &peeked) -> bool {
      if constexpr (!kSC) return take(i, r);
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        r.d[q] = peeked.d[q];
        r.jx[q] = peeked.jx[q];
        r.jy[q] = peeked.jy[q];
      }
      r.solid = peeked.solid;
      r.fluid = peeked.fluid;
      release();
      return true;
    };
    // reads the next ring row i (the one after the last taken) into `r`
    // without releasing its stage (kSC: the row above the source row being
    // taken); false on a timeout
    auto peek = [&](int i, Row &r) -> bool {
      return __all_sync(kFull, fetch(i, tst, tph, r));
    };
    int failed = -1;
    // potential terms of two rows (kSC), swapping roles row by row
    float2 tC0[kP], tA0[kP], tS0[kP], tC1[kP], tA1[kP], tS1[kP];
    Row rn;  // kSC: the row above the current source row
    if constexpr (kSC) {
      // the row below the first source row and the first source row itself
      if (!take(0, rb)) {
        failed = 0;
      } else if (!peek(1, rn)) {
        failed = 1;
      } else {
        psi_terms(rb, tC0, tA0, tS0);
        psi_terms(rn, tC1, tA1, tS1);
#pragma unroll
        for (int q = 0; q < kP; ++q) rb.zx[q] = rb.zy[q] = bc(0.f);
      }
    }
    if constexpr (!kClean && !kSC) {
      // the general code: one row per loop turn (half the loop's code), the
      // row just computed copied into the previous-row buffer
#pragma unroll 1
      for (int i = 0; i < 2 * npairs; ++i) {
        if (!take(i, ra)) {
          failed = i;
          break;
        }
        row(i, ra, rb, rn, tC0, tA0, tS0, tC1, tA1, tS1);
        rb = ra;
      }
    }
    // kSC: every source row was peeked as the row above the one before it
    // (the first one before the loop), so it is taken from the registers
    for (int k = 0; (kClean || kSC) && k < npairs && failed < 0; ++k) {
      const int r0 = 2 * k + kLead;  // ring row of source row 2k
      if (!take_peeked(r0, ra, rn)) {
        failed = r0;
        break;
      }
      if (kSC && !peek(r0 + 1, rn)) {
        failed = r0 + 1;
        break;
      }
      row(2 * k, ra, rb, rn, tC0, tA0, tS0, tC1, tA1, tS1);
      if (!take_peeked(r0 + 1, rb, rn)) {
        failed = r0 + 1;
        break;
      }
      if (kSC && !peek(r0 + 2, rn)) {
        failed = r0 + 2;
        break;
      }
      row(2 * k + 1, rb, ra, rn, tC1, tA1, tS1, tC0, tA0, tS0);
    }
    if (failed >= 0) {
      if (lane == 0) atomicOr(a.flag, kFlagCopyTimeout);
      // let every copy still in flight land before the warp leaves its ring
      for (int i = failed; i < issued; ++i) {
        if (source_row(i) < 0) continue;
        const unsigned ui = static_cast<unsigned>(i);
        mbar_wait(bars + ui % kS, (ui / kS) & 1u);
      }
    }
    // release the barriers so the ring can serve another tile
    __syncwarp();
    if (lane == 0)
      for (int st = 0; st < kS; ++st) mbar_inval(bars + st);
    __syncwarp();
  }

  if constexpr (kReduce) {
    if (!owner) {  // a halo lane's sums (clean tiles add every lane's)
      rs_num = rs_den = bc(0.f);
      rs_mass = rs_comp = 0.f;
      rmin = 1.0f;
    }
    double v0 = static_cast<double>(rs_num.x) + rs_num.y;
    double v1 = static_cast<double>(rs_den.x) + rs_den.y;
    double v2 = static_cast<double>(rs_mass) - rs_comp;
#pragma unroll
    for (int o = kLanes / 2; o > 0; o >>= 1) {
      v0 += __shfl_xor_sync(kFull, v0, o);
      v1 += __shfl_xor_sync(kFull, v1, o);
      v2 += __shfl_xor_sync(kFull, v2, o);
    }
    const bool bad = !(rmin > 0.f) || !isfinite(v0) || !isfinite(v1) ||
                     !isfinite(v2);
    const bool any_bad = __any_sync(kFull, bad);
    if (lane == 0) {
      double *q = a.partials + 3 * ((by * gx + bx) * kWarps + w);
      q[0] = v0;
      q[1] = v1;
      q[2] = v2;
      if (any_bad) atomicOr(a.flag, kFlagUnstable);
    }
  }
}

// Runs warp tile (bx, by, w).  kDual: with the code for clean tiles when
// the tile's flag says so (flags absent: the general code); otherwise the
// general code only, which keeps the kernel's registers for one code path.
template <typename T, int kC, int kRows, int kS, bool kReduce, bool kDual,
          bool kSC = false>
__device__ __forceinline__ void run_tile(const StepLaunch &a, int64_t bx,
                                         int64_t by, int w, int slot,
                                         int64_t gx, const SolidSums *lut,
                                         unsigned char *smem) {
  if constexpr (!kDual) {
    step_tile<T, kC, kRows, kS, kReduce, false, kSC>(a, bx, by, w, slot, gx,
                                                     lut, smem);
    return;
  }
  const bool clean = a.clean && a.clean[(by * gx + bx) * kWarps + w];
  if (clean)
    step_tile<T, kC, kRows, kS, kReduce, true>(a, bx, by, w, slot, gx, lut,
                                               smem);
  else
    step_tile<T, kC, kRows, kS, kReduce, false>(a, bx, by, w, slot, gx, lut,
                                                smem);
}

// kSC: the Shan-Chen multiphase step (general tile code only: the clean-tile
// test does not cover the extra rows its force needs).
template <typename T, int kC, int kRows, int kMinBlocks, int kS, bool kReduce,
          bool kDual, bool kSC = false>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    lbm_step_kernel(const StepLaunch a) {
  static_assert(!(kDual && kSC), "the multiphase step has no clean-tile code");
  extern __shared__ __align__(128) unsigned char smem[];
  SolidSums *lut = reinterpret_cast<SolidSums *>(smem);
  build_solid_lut(lut);
  __syncthreads();
  const int warp = threadIdx.x / kLanes;
  run_tile<T, kC, kRows, kS, kReduce, kDual, kSC>(
      a, blockIdx.x, blockIdx.y, warp, warp, gridDim.x, lut, smem);
}

// The launch state of batch member m for one step: copy c holds its state.
__device__ __forceinline__ void fill_launch(StepLaunch &a, const BatchMember &m,
                                            int c, int storage,
                                            unsigned clock) {
  StepLaunch t;  // the defaults (wait limit, single phase, ...) included
  t.src = m.f[c];
  t.dst = m.f[1 - c];
  t.mask = m.mask;
  t.nx = m.nx;
  t.ny = m.ny;
  t.pitch = m.pitch;
  t.periodic_x = m.periodic_x;
  t.periodic_y = m.periodic_y;
  t.fx = m.fx;
  t.fy = m.fy;
  t.partials = m.partials;
  t.flag = m.flag;
  t.storage = storage;
  t.sr = m.sr;
  t.step = static_cast<uint32_t>(m.step_base) + clock;
  t.clean = m.clean;
  a = t;
}

// Batched step: a persistent grid whose warps take warp tiles of many domains
// from one work list through an atomic counter, so that one launch advances
// every member of a batch by one step.  Each warp works on its own (its own
// ring, no block barrier between tiles), and tile for tile it runs the same
// code as the single-domain kernel, so each member's result does not depend
// on the batch.
template <typename T, int kC, int kRows, int kMinBlocks, int kS, bool kReduce,
          bool kDual>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    lbm_batch_kernel(const BatchLaunch b) {
  extern __shared__ __align__(128) unsigned char smem[];
  SolidSums *lut = reinterpret_cast<SolidSums *>(smem);
  build_solid_lut(lut);
  // the batch clock: read by every block before the last block advances it
  const unsigned clock = *b.clock;
  __syncthreads();
  const int n = *b.nitems;
  const int slot = threadIdx.x / kLanes;
  const bool lead = (threadIdx.x & (kLanes - 1)) == 0;
  // The item's launch state lives in the warp's shared-memory slot, not in
  // registers: the tile code reads its fields where it needs them, which
  // keeps the kernel inside the register budget of three blocks per SM.
  StepLaunch &a = reinterpret_cast<StepLaunch *>(
      smem + smem_bytes<T, kC, kS>())[slot];
  for (;;) {
    int it = 0;
    if (lead) it = static_cast<int>(atomicAdd(b.counter, 1u));
    it = __shfl_sync(kFull, it, 0);
    if (it >= n) break;
    __syncwarp();  // every lane is done with the previous item's state
    if (lead) {
      const int4 w = b.items[it];  // member, tile x, tile y, warp
      const BatchMember &m = b.members[w.x];
      const int c = (m.cur ^ b.parity) & 1;
      fill_launch(a, m, c, b.storage, clock);
    }
    __syncwarp();
    const int4 w = b.items[it];
    run_tile<T, kC, kRows, kS, kReduce, kDual>(
        a, w.y, w.z, w.w, slot, b.members[w.x].gx, lut, smem);
  }
  // the last block to finish advances the clock for the next launch (every
  // thread read it before its block's first tile)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(b.done, 1u) == gridDim.x - 1) {
      *b.done = 0u;
      *b.clock = clock + 1u;
      __threadfence();
    }
  }
}

template <typename T>
__global__ void pack_kernel(const double *__restrict__ staging, Fields f,
                            int64_t nx, int64_t pitch, int64_t y0,
                            int64_t rows) {
  using S = Storage<T>;
  const int64_t n = nx * rows;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t y = y0 + i / nx, x = i % nx;
    const int64_t o = y * pitch + x;
    static_cast<T *>(f.d)[o] =
        S::encode(static_cast<float>(staging[i] - 1.0) * S::kD);
    static_cast<T *>(f.jx)[o] =
        S::encode(static_cast<float>(staging[n + i]) * S::kJ);
    static_cast<T *>(f.jy)[o] =
        S::encode(static_cast<float>(staging[2 * n + i]) * S::kJ);
  }
}

template <typename T>
__global__ void unpack_kernel(Fields f, const uint8_t *__restrict__ mask,
                              double *__restrict__ staging, int64_t nx,
                              int64_t pitch, int64_t y0, int64_t rows) {
  using S = Storage<T>;
  const int64_t n = nx * rows;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t y = y0 + i / nx, x = i % nx;
    const int64_t o = y * pitch + x;
    const bool solid = mask[o] == 1u;  // holds no fluid state: report rest
    const float d = S::decode(static_cast<const T *>(f.d)[o]) * (1.0f / S::kD);
    const float jx = S::decode(static_cast<const T *>(f.jx)[o]) * (1.0f / S::kJ);
    const float jy = S::decode(static_cast<const T *>(f.jy)[o]) * (1.0f / S::kJ);
    staging[i] = solid ? 1.0 : 1.0 + static_cast<double>(d);
    staging[n + i] = solid ? 0.0 : static_cast<double>(jx);
    staging[2 * n + i] = solid ? 0.0 : static_cast<double>(jy);
  }
}

// The change of the velocity field since a snapshot: per warp, the FP64
// sums of |u_now - u_snap|^2 and |u_now|^2 over fluid nodes (u = j / rho
// decoded from either copy), written as the first two of its partial triple
// (4 warps per block: the layout finalize_kernel sums).
template <typename T>
__global__ void __launch_bounds__(128)
    change_kernel(Fields now, Fields snap, const uint8_t *__restrict__ mask,
                  int64_t nx, int64_t ny, int64_t pitch,
                  double *__restrict__ partials) {
  using S = Storage<T>;
  double s0 = 0.0, s1 = 0.0;
  const int64_t n = nx * ny;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = (i / nx) * pitch + i % nx;
    if (mask[o] != 0u) continue;
    auto u_of = [&](const Fields &f, double &ux, double &uy) {
      const double rho =
          1.0 + S::decode(static_cast<const T *>(f.d)[o]) * (1.0 / S::kD);
      ux = S::decode(static_cast<const T *>(f.jx)[o]) * (1.0 / S::kJ) / rho;
      uy = S::decode(static_cast<const T *>(f.jy)[o]) * (1.0 / S::kJ) / rho;
    };
    double ax, ay, bx, by;
    u_of(now, ax, ay);
    u_of(snap, bx, by);
    s0 += (ax - bx) * (ax - bx) + (ay - by) * (ay - by);
    s1 += ax * ax + ay * ay;
  }
#pragma unroll
  for (int m = kLanes / 2; m > 0; m >>= 1) {
    s0 += __shfl_xor_sync(kFull, s0, m);
    s1 += __shfl_xor_sync(kFull, s1, m);
  }
  if ((threadIdx.x & (kLanes - 1)) == 0) {
    double *q = partials + 3 * (blockIdx.x * 4 + threadIdx.x / kLanes);
    q[0] = s0;
    q[1] = s1;
    q[2] = 0.0;
  }
}

// Writes the solid-node storage values rho - 1 = 0, j = -F.
template <typename T>
__global__ void solid_storage_kernel(Fields f, const uint8_t *__restrict__ mask,
                                     int64_t n, float fx, float fy) {
  using S = Storage<T>;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (mask[i] == 1u) {
      static_cast<T *>(f.d)[i] = S::encode(0.0f);
      static_cast<T *>(f.jx)[i] = S::encode(-fx * S::kJ);
      static_cast<T *>(f.jy)[i] = S::encode(-fy * S::kJ);
    }
  }
}

// Tile variants: columns per lane, output rows per warp, resident blocks per
// SM requested from the register allocator, shared-memory ring stages.
struct Variant {
  int cols, rows, min_blocks, stages;
  bool dual;  // also carries the clean-tile code (flags per warp tile)
};
constexpr Variant kVariants[] = {
    {4, 64, 3, 6, false}, {4, 32, 3, 6, false}, {4, 16, 3, 6, false},
    {4, 8, 3, 6, false},  {4, 64, 3, 6, true}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// Calls f(std::integral_constant<int, v>) for a run-time variant index v
// (variant 0 for an index out of range).
template <int kV = 0, typename F>
auto with_variant(int v, F &&f) {
  if constexpr (kV + 1 < kNumVariants) {
    if (v == kV) return f(std::integral_constant<int, kV>{});
    return with_variant<kV + 1>(v, static_cast<F &&>(f));
  } else {
    if (v == kV) return f(std::integral_constant<int, kV>{});
    return f(std::integral_constant<int, 0>{});
  }
}

// A variant forced through LBMTAU1_STEP_VARIANT (tuning), or -1.
int forced_variant() {
  static int v = [] {
    const char *e = getenv("LBMTAU1_STEP_VARIANT");
    int i = e ? atoi(e) : -1;
    return (i >= 0 && i < kNumVariants) ? i : -1;
  }();
  return v;
}

int active_variant() {
  const int f = forced_variant();
  return f >= 0 ? f : 0;
}

dim3 step_grid(int64_t nx, int64_t ny, int vi) {
  const Variant v = kVariants[(vi >= 0 && vi < kNumVariants) ? vi : 0];
  const int64_t tile_x = (kLanes - 2) * v.cols;
  const int64_t tile_y = static_cast<int64_t>(kWarps) * v.rows;
  const int64_t gx = (nx + tile_x - 1) / tile_x;
  const int64_t gy = (ny + tile_y - 1) / tile_y;
  return dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy), 1);
}

template <typename T, int kV, bool kReduce, bool kSC>
cudaError_t launch_kernel(const StepLaunch &a, dim3 g, cudaStream_t s) {
  constexpr Variant v = kVariants[kV];
  constexpr int smem = smem_bytes<T, v.cols, v.stages>();
  static_assert(smem <= 227 * 1024, "shared memory per block");
  auto kern = lbm_step_kernel<T, v.cols, v.rows, v.min_blocks, v.stages,
                              kReduce, v.dual && !kSC, kSC>;
  static cudaError_t attr = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  (void)cudaGetLastError();  // an earlier, unrelated non-sticky error
  kern<<<g, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// The variant's kernel; a nonzero multiphase coupling (FP32 storage only)
// takes the multiphase kernel of the same tile shape.
template <typename T, int kV, bool kReduce>
cudaError_t launch_variant(const StepLaunch &a, dim3 g, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value)
    if (a.g_sc != 0.0f) return launch_kernel<T, kV, kReduce, true>(a, g, s);
  return launch_kernel<T, kV, kReduce, false>(a, g, s);
}

template <typename T, bool kReduce>
cudaError_t launch_any(const StepLaunch &a, dim3 g, cudaStream_t s) {
  return with_variant(a.variant, [&](auto kv) {
    return launch_variant<T, decltype(kv)::value, kReduce>(a, g, s);
  });
}

// Resident blocks per SM of a variant's (unreduced) step kernel.
template <typename T, int kV>
int occupancy_of() {
  constexpr Variant v = kVariants[kV];
  constexpr int smem = smem_bytes<T, v.cols, v.stages>();
  auto kern =
      lbm_step_kernel<T, v.cols, v.rows, v.min_blocks, v.stages, false, v.dual>;
  static int occ = [&] {
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads,
                                                      smem) != cudaSuccess)
      n = 0;
    return n;
  }();
  return occ;
}

template <typename T>
int occupancy(int v) {
  return with_variant(v, [](auto kv) {
    return occupancy_of<T, decltype(kv)::value>();
  });
}

// Picks the variant with the shortest expected step time for an nx x ny
// domain.  The model, fitted to step times measured on a GB300 (periodic
// boxes and cavities, 1024^2 .. 16384^2): blocks are spread evenly over the
// SMs, so the busiest SM runs ceil(blocks / SMs) of them, up to the kernel's
// occupancy at a time; one block costs the kRows + 2 source rows each of its
// warps marches; and k blocks resident together get through their rows
// kConcurrent[k] times as fast as one block alone (the kernel is issue- and
// latency-bound: more resident warps hide more latency).  A last, partial
// round of blocks runs at its own, lower rate.
template <typename T>
int choose_variant_t(int64_t nx, int64_t ny) {
  constexpr double kConcurrent[] = {1.0, 1.0, 1.3, 1.58};
  static int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess)
      n = 0;
    return n;
  }();
  if (sms <= 0) return 0;
  int best = 0;
  double best_time = 0.0;
  for (int i = 0; i < kNumVariants; ++i) {
    const Variant v = kVariants[i];
    if (v.dual) continue;  // chosen only through dual_variant, by its flags
    const int occ = occupancy<T>(i);
    if (occ <= 0) continue;
    const dim3 g = step_grid(nx, ny, i);
    const int64_t blocks = static_cast<int64_t>(g.x) * g.y;
    const int64_t per_sm = (blocks + sms - 1) / sms;
    const int64_t k = occ < 3 ? occ : 3;
    const int64_t full = per_sm / k, rest = per_sm % k;
    const double t = (v.rows + 2.0) * (static_cast<double>(full * k) /
                                           kConcurrent[k] +
                                       static_cast<double>(rest) /
                                           kConcurrent[rest]);
    if (best_time == 0.0 || t < best_time * (1.0 - 1e-9)) {
      best_time = t;
      best = i;
    }
  }
  return best;
}

template <typename T, int kV, bool kReduce>
cudaError_t launch_batch_variant(const BatchLaunch &b, cudaStream_t s) {
  constexpr Variant v = kVariants[kV];
  constexpr int smem = batch_smem_bytes<T, v.cols, v.stages>();
  static_assert(smem <= 227 * 1024, "shared memory per block");
  auto kern =
      lbm_batch_kernel<T, v.cols, v.rows, v.min_blocks, v.stages, kReduce,
                       v.dual>;
  // persistent grid: every resident block slot of the device, computed once
  static int grid = [&] {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
      return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads,
                                                      smem) != cudaSuccess)
      return 0;
    return sms * (per_sm > 0 ? per_sm : 1);
  }();
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  (void)cudaGetLastError();
  kern<<<grid, kThreads, smem, s>>>(b);
  return cudaGetLastError();
}

template <typename T, bool kReduce>
cudaError_t launch_batch_any(int v, const BatchLaunch &b, cudaStream_t s) {
  return with_variant(v, [&](auto kv) {
    return launch_batch_variant<T, decltype(kv)::value, kReduce>(b, s);
  });
}

template <typename T>
cudaError_t launch_step_t(const StepLaunch &a, bool reduce, cudaStream_t s) {
  const dim3 g = step_grid(a.nx, a.ny, a.variant);
  return reduce ? launch_any<T, true>(a, g, s) : launch_any<T, false>(a, g, s);
}

template <typename T>
cudaError_t launch_batch_t(int v, const BatchLaunch &b, bool reduce,
                           cudaStream_t s) {
  return reduce ? launch_batch_any<T, true>(v, b, s)
                : launch_batch_any<T, false>(v, b, s);
}


int copy_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return static_cast<int>(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

template <typename T>
cudaError_t pack_t(const double *staging, Fields f, int64_t nx, int64_t pitch,
                   int64_t y0, int64_t rows, cudaStream_t s) {
  (void)cudaGetLastError();
  pack_kernel<T><<<copy_grid(nx * rows), 256, 0, s>>>(staging, f, nx, pitch,
                                                      y0, rows);
  return cudaGetLastError();
}
template <typename T>
cudaError_t unpack_t(Fields f, const uint8_t *mask, double *staging,
                     int64_t nx, int64_t pitch, int64_t y0, int64_t rows,
                     cudaStream_t s) {
  (void)cudaGetLastError();
  unpack_kernel<T><<<copy_grid(nx * rows), 256, 0, s>>>(f, mask, staging, nx,
                                                        pitch, y0, rows);
  return cudaGetLastError();
}
template <typename T>
cudaError_t solid_t(Fields f, const uint8_t *mask, int64_t n, float fx,
                    float fy, cudaStream_t s) {
  (void)cudaGetLastError();
  solid_storage_kernel<T><<<copy_grid(n), 256, 0, s>>>(f, mask, n, fx, fy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t change_t(Fields now, Fields snap, const uint8_t *mask, int64_t nx,
                     int64_t ny, int64_t pitch, double *partials,
                     int64_t blocks, cudaStream_t s) {
  (void)cudaGetLastError();
  change_kernel<T><<<static_cast<unsigned>(blocks), 128, 0, s>>>(
      now, snap, mask, nx, ny, pitch, partials);
  return cudaGetLastError();
}

// The launchers of storage type T, as the table lbm_step.cu dispatches on.
template <typename T>
constexpr StorageOps make_ops() {
  return StorageOps{&launch_step_t<T>, &launch_batch_t<T>, &choose_variant_t<T>,
                    &pack_t<T>,        &unpack_t<T>,       &solid_t<T>,
                    &change_t<T>};
}

}  // namespace
}  // namespace lbmtau1
