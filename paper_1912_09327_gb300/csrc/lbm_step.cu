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
// Arithmetic form.  The device stores delta = rho - 1 and j in FP32.  With
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
// Kernel structure (HBM-bound stencil; no tensor cores).  A warp owns a tile
// of 120 columns x 32 rows.  Lane l holds the four columns x0 - 4 + 4l ..
// x0 - 1 + 4l as one float4 per field, so lanes 1..30 own the 120 outputs and
// lanes 0 and 31 carry the one-column halos (coalesced 512-byte row segments,
// 16-byte aligned because rows are padded to 32 nodes).  The warp marches
// down its tile one source row at a time: each source row is read from HBM
// once, turned into per-node quantities once (one reciprocal per node), the
// left/right neighbour columns are exchanged with warp shuffles, and the row's
// contributions are added to the three output rows it feeds (above, same,
// below).  The output row above is then complete and is stored as float4.
// The next source row is prefetched into registers while the current one is
// processed.  Four warps per block stack vertically so that the shared halo
// rows hit in L1/L2.  Periodic edges and ragged tails take a per-column path.
// On the last step of an lbm_step call the same kernel also reduces
// sum |du|^2, sum |u|^2 and sum delta (warp shuffles, FP64 block partials) and
// raises a sticky flag on rho <= 0 or non-finite values.
#include <float.h>
#include <stdint.h>

#include "lbm_step.cuh"

namespace lbmtau1 {
namespace {

constexpr int kLanes = 32;
constexpr int kCols = 4;                      // columns per lane (one float4)
constexpr int kTileX = (kLanes - 2) * kCols;  // 120 output columns per warp
constexpr int kWarps = 4;                     // warps per block, stacked in y
constexpr int kRowsPerWarp = 32;              // output rows per warp
constexpr int kThreads = kWarps * kLanes;
constexpr unsigned kFull = 0xffffffffu;

// D2Q9 weights (rest 4/9, axis 1/9, diagonal 1/36) and the combinations of
// them that appear in the closed form.
constexpr float k4_9 = 4.0f / 9.0f;
constexpr float k1_9 = 1.0f / 9.0f;
constexpr float k1_36 = 1.0f / 36.0f;
constexpr float k1_12 = 1.0f / 12.0f;  // 3 * (1/36)
constexpr float k1_3 = 1.0f / 3.0f;    // 3 * (1/9)
constexpr float k1_6 = 1.0f / 6.0f;    // 2 * (1/12)

__device__ __forceinline__ float comp(const float4 &v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

__device__ __forceinline__ int64_t wrap_index(int64_t v, int64_t n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// One source row as loaded: four columns of raw fields and their node types.
struct RawRow {
  float4 d, jx, jy;
  unsigned solid;  // bit j: column j is solid or outside a non-periodic edge
  unsigned fluid;  // bit j: column j is a fluid node
};

__device__ __forceinline__ unsigned byte_bits(unsigned v) {
  // gathers bit 0 of each byte into bits 0..3
  v &= 0x01010101u;
  return (v | (v >> 7) | (v >> 14) | (v >> 21)) & 0xFu;
}

__device__ __forceinline__ void load_row(const StepLaunch &a, int64_t r,
                                         int64_t xb, RawRow &o) {
  o.d = o.jx = o.jy = make_float4(0.f, 0.f, 0.f, 0.f);
  o.solid = 0xFu;
  o.fluid = 0u;
  if (r < 0 || r >= a.ny) {
    if (!a.periodic_y) return;  // outside a wall-less edge: solid
    r = wrap_index(r, a.ny);
  }
  const int64_t row = r * a.pitch;
  if (xb >= 0 && xb + kCols <= a.nx) {
    o.d = __ldg(reinterpret_cast<const float4 *>(a.src.d + row + xb));
    o.jx = __ldg(reinterpret_cast<const float4 *>(a.src.jx + row + xb));
    o.jy = __ldg(reinterpret_cast<const float4 *>(a.src.jy + row + xb));
    const unsigned m =
        __ldg(reinterpret_cast<const unsigned *>(a.mask + row + xb));
    o.solid = byte_bits(m);                   // type 1 has bit 0 set
    o.fluid = byte_bits(~(m | (m >> 1)));     // type 0 has bits 0, 1 clear
    return;
  }
  float dv[kCols], xv[kCols], yv[kCols];
  unsigned solid = 0u, fluid = 0u;
#pragma unroll
  for (int j = 0; j < kCols; ++j) {
    int64_t x = xb + j;
    bool in = x >= 0 && x < a.nx;
    if (!in && a.periodic_x) {
      x = wrap_index(x, a.nx);
      in = true;
    }
    dv[j] = xv[j] = yv[j] = 0.f;
    if (in) {
      dv[j] = __ldg(a.src.d + row + x);
      xv[j] = __ldg(a.src.jx + row + x);
      yv[j] = __ldg(a.src.jy + row + x);
      const unsigned t = __ldg(a.mask + row + x);
      solid |= (t == 1u) << j;
      fluid |= (t == 0u) << j;
    } else {
      solid |= 1u << j;
    }
  }
  o.d = make_float4(dv[0], dv[1], dv[2], dv[3]);
  o.jx = make_float4(xv[0], xv[1], xv[2], xv[3]);
  o.jy = make_float4(yv[0], yv[1], yv[2], yv[3]);
  o.solid = solid;
  o.fluid = fluid;
}

// Partial sums of the three moments for one output row (this lane's columns).
struct Acc {
  float dd[kCols], mx[kCols], my[kCols];
};

template <bool kReduce>
__global__ void __launch_bounds__(kThreads, 3)
    lbm_step_kernel(const StepLaunch a) {
  const int lane = threadIdx.x & (kLanes - 1);
  const int warp = threadIdx.x / kLanes;
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * kTileX;
  const int64_t xb = x0 - kCols + static_cast<int64_t>(kCols) * lane;
  const int64_t y0 =
      (static_cast<int64_t>(blockIdx.y) * kWarps + warp) * kRowsPerWarp;
  const int64_t y1 = min(y0 + kRowsPerWarp, a.ny);
  const bool owner = lane >= 1 && lane <= kLanes - 2 && xb < a.nx;
  const float fx = a.fx, fy = a.fy;

  float num = 0.f, den = 0.f, mass = 0.f;
  bool bad = false;

  if (y0 < a.ny) {
    Acc accA, accB;  // output rows r-1 and r while source row r arrives
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      accA.dd[j] = accA.mx[j] = accA.my[j] = 0.f;
      accB.dd[j] = accB.mx[j] = accB.my[j] = 0.f;
    }
    float zpx[kCols], zpy[kCols];  // z of row r-2 (D row of output r-1)
    float zcx[kCols], zcy[kCols];  // z of row r-1
    float hd[kCols], hx[kCols], hy[kCols];  // raw fields of row r-1
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      zpx[j] = zpy[j] = zcx[j] = zcy[j] = 0.f;
      hd[j] = hx[j] = hy[j] = 0.f;
    }
    unsigned sD6 = 0u, sO6 = 0u;  // solid bits (cols -1..4) of rows r-2, r-1
    unsigned fluidO = 0u;         // fluid bits of row r-1

    RawRow cur;
    load_row(a, y0 - 1, xb, cur);
    for (int64_t r = y0 - 1; r <= y1; ++r) {
      RawRow nxt;
      if (r < y1) load_row(a, r + 1, xb, nxt);

      // Per-node quantities of source row r, own columns (index j + 1).
      float df[kCols + 2], zx[kCols + 2], zy[kCols + 2];
      float A[kCols + 2], G[kCols + 2], X[kCols + 2];
      float B[kCols], R0[kCols];
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        const bool s = (cur.solid >> j) & 1u;
        const float d = comp(cur.d, j);
        const float zxj = s ? -fx : comp(cur.jx, j);
        const float zyj = s ? -fy : comp(cur.jy, j);
        const float mx = zxj + fx;  // j + F, exactly 0 on solid nodes
        const float my = zyj + fy;
        const float dfj = s ? 0.f : d;
        const float ir = __frcp_rn(1.0f + dfj);
        const float t = mx * ir;
        const float pxx = t * mx, pxy = t * my, pyy = my * my * ir;
        const float tr = pxx + pyy;
        df[j + 1] = dfj;
        zx[j + 1] = zxj;
        zy[j + 1] = zyj;
        A[j + 1] = 3.0f * pxx - 1.5f * pyy;
        B[j] = 3.0f * pyy - 1.5f * pxx;
        G[j + 1] = fmaf(3.0f, tr, dfj);
        X[j + 1] = 9.0f * pxy;
        R0[j] = fmaf(-1.5f, tr, d);
      }
      // Halo columns -1 and 4 from the neighbouring lanes.
      df[0] = __shfl_up_sync(kFull, df[kCols], 1);
      zx[0] = __shfl_up_sync(kFull, zx[kCols], 1);
      zy[0] = __shfl_up_sync(kFull, zy[kCols], 1);
      A[0] = __shfl_up_sync(kFull, A[kCols], 1);
      G[0] = __shfl_up_sync(kFull, G[kCols], 1);
      X[0] = __shfl_up_sync(kFull, X[kCols], 1);
      df[kCols + 1] = __shfl_down_sync(kFull, df[1], 1);
      zx[kCols + 1] = __shfl_down_sync(kFull, zx[1], 1);
      zy[kCols + 1] = __shfl_down_sync(kFull, zy[1], 1);
      A[kCols + 1] = __shfl_down_sync(kFull, A[1], 1);
      G[kCols + 1] = __shfl_down_sync(kFull, G[1], 1);
      X[kCols + 1] = __shfl_down_sync(kFull, X[1], 1);
      const unsigned sl = __shfl_up_sync(kFull, cur.solid, 1);
      const unsigned sr = __shfl_down_sync(kFull, cur.solid, 1);
      const unsigned s6 = ((sl >> (kCols - 1)) & 1u) | (cur.solid << 1) |
                          ((sr & 1u) << (kCols + 1));

      Acc accC;
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        const int L = j, C = j + 1, R = j + 2;
        const float mxL = zx[L] + fx, mxR = zx[R] + fx;
        const float myL = zy[L] + fy, myR = zy[R] + fy, myC = zy[C] + fy;
        const float hxl = zx[L] - zx[C], hxr = zx[R] - zx[C];  // exact
        const float hyl = zy[L] - zy[C], hyr = zy[R] - zy[C];
        // row r as the row above output row r-1 (NW, U, NE)
        accA.dd[j] += k1_9 * (df[C] - 3.0f * myC + B[j]) +
                      k1_36 * (G[L] + G[R] + 3.0f * (mxL - myL) -
                               3.0f * (mxR + myR) - X[L] + X[R]);
        accA.mx[j] += k1_36 * (G[L] - G[R] - X[L] - X[R]) +
                      k1_12 * ((myR - myL) + (hxl + hxr));
        accA.my[j] += -k1_9 * (df[C] + B[j]) +
                      k1_36 * (X[L] - X[R] - G[L] - G[R]) +
                      k1_12 * ((mxR - mxL) + (hyl + hyr));
        // row r as the same row of output row r (L, O, R)
        accB.dd[j] += k4_9 * R0[j] +
                      k1_9 * (df[L] + df[R] + 3.0f * (mxL - mxR) + A[L] + A[R]);
        accB.mx[j] +=
            k1_9 * (df[L] - df[R] + A[L] - A[R]) + k1_3 * (hxl + hxr);
        // row r as the row below output row r+1 (SW, D, SE)
        accC.dd[j] = k1_9 * (df[C] + 3.0f * myC + B[j]) +
                     k1_36 * (G[L] + G[R] + 3.0f * (mxL + myL) +
                              3.0f * (myR - mxR) + X[L] - X[R]);
        accC.mx[j] = k1_36 * (G[L] - G[R] + X[L] + X[R]) +
                     k1_12 * ((myL - myR) + (hxl + hxr));
        accC.my[j] = k1_9 * (df[C] + B[j]) +
                     k1_36 * (G[L] + G[R] + X[L] - X[R]) +
                     k1_12 * ((mxL - mxR) + (hyl + hyr));
      }

      // Output row r-1 is complete: rows r-2 (D), r-1 (O), r (U).
      const int64_t yo = r - 1;
      const bool any_solid = __any_sync(kFull, (sD6 | sO6 | s6) != 0u);
      float4 od, ox, oy;
      float outd[kCols], outx[kCols], outy[kCols];
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        float S0 = 0.f, Sx = 0.f, Sy = 0.f;  // sums of w_k (1, c_k) over solid P
        if (any_solid) {
          const float sL = (sO6 >> j) & 1u, sR = (sO6 >> (j + 2)) & 1u;
          const float sD = (sD6 >> (j + 1)) & 1u, sU = (s6 >> (j + 1)) & 1u;
          const float sSW = (sD6 >> j) & 1u, sSE = (sD6 >> (j + 2)) & 1u;
          const float sNW = (s6 >> j) & 1u, sNE = (s6 >> (j + 2)) & 1u;
          S0 = k1_9 * ((sL + sR) + (sD + sU)) +
               k1_36 * ((sSW + sSE) + (sNW + sNE));
          Sx = k1_9 * (sL - sR) + k1_36 * ((sSW - sSE) + (sNW - sNE));
          Sy = k1_9 * (sD - sU) + k1_36 * ((sSW + sSE) - (sNW + sNE));
        }
        const float dO = hd[j], jxO = hx[j], jyO = hy[j];
        const float dn = fmaf(dO, S0, accA.dd[j]);
        const float mxn =
            jxO + (fx + accA.mx[j] +
                   k1_6 * ((zpx[j] - jxO) + (zx[j + 1] - jxO)) + dO * Sx);
        const float myn =
            jyO + (fy + accA.my[j] + 0.5f * ((zpy[j] - jyO) + (zy[j + 1] - jyO)) +
                   dO * Sy);
        const bool upd = (fluidO >> j) & 1u;
        outd[j] = upd ? dn : dO;
        outx[j] = upd ? mxn : jxO;
        outy[j] = upd ? myn : jyO;
        if (kReduce) {
          if (upd && owner && yo >= y0 && xb + j < a.nx) {
            const float rn = 1.0f + dn;
            bad |= !(rn > 0.f) || !(fabsf(mxn) <= FLT_MAX) ||
                   !(fabsf(myn) <= FLT_MAX);
            const float ro = 1.0f + dO;
            const float uxo = jxO / ro, uyo = jyO / ro;
            const float uxn = mxn / rn, uyn = myn / rn;
            const float ddx = uxn - uxo, ddy = uyn - uyo;
            num = fmaf(ddx, ddx, fmaf(ddy, ddy, num));
            den = fmaf(uxn, uxn, fmaf(uyn, uyn, den));
            mass += dn;
          }
        }
      }
      if (owner && yo >= y0) {
        od = make_float4(outd[0], outd[1], outd[2], outd[3]);
        ox = make_float4(outx[0], outx[1], outx[2], outx[3]);
        oy = make_float4(outy[0], outy[1], outy[2], outy[3]);
        const int64_t o = yo * a.pitch + xb;
        *reinterpret_cast<float4 *>(a.dst.d + o) = od;
        *reinterpret_cast<float4 *>(a.dst.jx + o) = ox;
        *reinterpret_cast<float4 *>(a.dst.jy + o) = oy;
      }

      // Shift the window by one row.
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        accA.dd[j] = accB.dd[j];
        accA.mx[j] = accB.mx[j];
        accA.my[j] = accB.my[j];
        accB.dd[j] = accC.dd[j];
        accB.mx[j] = accC.mx[j];
        accB.my[j] = accC.my[j];
        zpx[j] = zcx[j];
        zpy[j] = zcy[j];
        zcx[j] = zx[j + 1];
        zcy[j] = zy[j + 1];
        hd[j] = comp(cur.d, j);
        hx[j] = comp(cur.jx, j);
        hy[j] = comp(cur.jy, j);
      }
      sD6 = sO6;
      sO6 = s6;
      fluidO = cur.fluid;
      if (r < y1) cur = nxt;
    }
  }

  if (kReduce) {
    __shared__ double part[kWarps][3];
    double v0 = num, v1 = den, v2 = mass;
#pragma unroll
    for (int o = kLanes / 2; o > 0; o >>= 1) {
      v0 += __shfl_xor_sync(kFull, v0, o);
      v1 += __shfl_xor_sync(kFull, v1, o);
      v2 += __shfl_xor_sync(kFull, v2, o);
    }
    const bool any_bad = __any_sync(kFull, bad);
    if (lane == 0) {
      part[warp][0] = v0;
      part[warp][1] = v1;
      part[warp][2] = v2;
      if (any_bad) atomicOr(a.flag, 1u);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += part[w][threadIdx.x];
      const int64_t b =
          static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[3 * b + threadIdx.x] = s;
    }
  }
}

constexpr int kFinalizeThreads = 512;

__global__ void __launch_bounds__(kFinalizeThreads)
    finalize_kernel(const double *__restrict__ partials, int64_t nblocks,
                    double *__restrict__ out) {
  __shared__ double buf[3][kFinalizeThreads];
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t b = threadIdx.x; b < nblocks; b += kFinalizeThreads)
    for (int k = 0; k < 3; ++k) s[k] += partials[3 * b + k];
  for (int k = 0; k < 3; ++k) buf[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = kFinalizeThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 3; ++k) buf[k][threadIdx.x] += buf[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = buf[threadIdx.x][0];
}

__global__ void pack_kernel(const double *__restrict__ staging, Fields f,
                            int64_t nx, int64_t pitch, int64_t y0,
                            int64_t rows) {
  const int64_t n = nx * rows;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t y = y0 + i / nx, x = i % nx;
    const int64_t o = y * pitch + x;
    f.d[o] = static_cast<float>(staging[i] - 1.0);
    f.jx[o] = static_cast<float>(staging[n + i]);
    f.jy[o] = static_cast<float>(staging[2 * n + i]);
  }
}

__global__ void unpack_kernel(Fields f, double *__restrict__ staging,
                              int64_t nx, int64_t pitch, int64_t y0,
                              int64_t rows) {
  const int64_t n = nx * rows;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t y = y0 + i / nx, x = i % nx;
    const int64_t o = y * pitch + x;
    staging[i] = 1.0 + static_cast<double>(f.d[o]);
    staging[n + i] = static_cast<double>(f.jx[o]);
    staging[2 * n + i] = static_cast<double>(f.jy[o]);
  }
}

dim3 step_grid(int64_t nx, int64_t ny) {
  const int64_t gx = (nx + kTileX - 1) / kTileX;
  const int64_t gy =
      (ny + kWarps * kRowsPerWarp - 1) / (kWarps * kRowsPerWarp);
  return dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy), 1);
}

int copy_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return static_cast<int>(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

int64_t step_blocks(int64_t nx, int64_t ny) {
  const dim3 g = step_grid(nx, ny);
  return static_cast<int64_t>(g.x) * g.y;
}

cudaError_t launch_step(const StepLaunch &a, bool reduce, cudaStream_t s) {
  const dim3 g = step_grid(a.nx, a.ny);
  if (reduce)
    lbm_step_kernel<true><<<g, kThreads, 0, s>>>(a);
  else
    lbm_step_kernel<false><<<g, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int64_t nblocks,
                            double *out, cudaStream_t s) {
  finalize_kernel<<<1, kFinalizeThreads, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double *staging, Fields f, int64_t nx,
                        int64_t pitch, int64_t y0, int64_t rows,
                        cudaStream_t s) {
  pack_kernel<<<copy_grid(nx * rows), 256, 0, s>>>(staging, f, nx, pitch, y0,
                                                   rows);
  return cudaGetLastError();
}

cudaError_t launch_unpack(Fields f, double *staging, int64_t nx, int64_t pitch,
                          int64_t y0, int64_t rows, cudaStream_t s) {
  unpack_kernel<<<copy_grid(nx * rows), 256, 0, s>>>(f, staging, nx, pitch, y0,
                                                     rows);
  return cudaGetLastError();
}

}  // namespace lbmtau1
