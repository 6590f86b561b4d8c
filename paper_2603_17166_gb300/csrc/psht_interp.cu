// Point side of the transform: theta* reduction, binning of the points into grid tiles, and the
// ES-kernel interpolation (gather, synthesis) and spreading (scatter-add, adjoint).
//
// A point at colatitude theta is mapped to Theta = pi beta/theta_max, beta = theta or pi - theta
// (Sec. II step 3), then to fine-grid coordinates t = Theta nTheta/2pi, u = (phi mod 2pi) nphi/2pi.
// Its window is rows r0 .. r0+W-1 and columns q0 .. q0+W-1 with r0 = ceil(t - W/2), q0 = ceil(u - W/2),
// and weights psi(2(t - r0 - i)/W) psi(2(u - q0 - k)/W), psi(z) = exp(beta_es (sqrt(1 - z^2) - 1))
// (the ES kernel of Barnett, Magland & af Klinteberg 2019, the NUFFT the paper defers to, Sec. I.B).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "psht_common.cuh"

namespace psht {

namespace {

constexpr int kBinThreads = 256;
constexpr int kInterpThreads = 256;

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// out[0] = max theta, out[1] = max (pi - theta), out[2] = count of invalid points (as bits/int)
__global__ void k_reduce(const double* __restrict__ theta, const double* __restrict__ phi, int64_t n,
                         unsigned long long* __restrict__ out) {
  double mN = 0.0, mS = 0.0;
  unsigned long long bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = theta[i], f = phi[i];
    if (!(t >= 0.0 && t <= M_PI) || !isfinite(f)) {
      ++bad;
      continue;
    }
    mN = fmax(mN, t);
    mS = fmax(mS, M_PI - t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mN = fmax(mN, __shfl_xor_sync(0xffffffffu, mN, o));
    mS = fmax(mS, __shfl_xor_sync(0xffffffffu, mS, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax(&out[0], dbits(mN));
    atomicMax(&out[1], dbits(mS));
    if (bad) atomicAdd(&out[2], bad);
  }
}

struct BinGeom {
  int pole;
  double theta_max, nTheta, nphi;
  int W, r_lo, padq, TR, TQ, ntr, ntq;
};

__device__ __forceinline__ void point_tu(const BinGeom& g, double th, double ph, double& t, double& u) {
  const double beta = g.pole > 0 ? th : M_PI - th;
  const double Th = beta * (M_PI / g.theta_max);
  t = Th * (g.nTheta / (2.0 * M_PI));
  const double pr = ph - 2.0 * M_PI * floor(ph / (2.0 * M_PI));
  u = pr * (g.nphi / (2.0 * M_PI));
  if (u >= g.nphi) u -= g.nphi;
  if (u < 0.0) u = 0.0;
}

// fine binning key of a point: tile (tr, tq) and base cell (lr, lq) inside it, so that sorting by
// the key groups points by tile and orders each tile's points by base cell
__global__ void k_bin_count(const double* __restrict__ theta, const double* __restrict__ phi, int64_t n, BinGeom g,
                            int* __restrict__ key_of, int* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double t, u;
    point_tu(g, theta[i], phi[i], t, u);
    const int r0 = (int)ceil(t - 0.5 * g.W), q0 = (int)ceil(u - 0.5 * g.W);
    const int dr = r0 - g.r_lo, dq = q0 + g.padq;
    if (dr < 0 || dq < 0 || dr / g.TR >= g.ntr || dq / g.TQ >= g.ntq) {  // outside the planned rows: reported
      key_of[i] = -1;
      continue;
    }
    const int tr = dr / g.TR, tq = dq / g.TQ;
    const int key = ((tr * g.ntq + tq) * g.TR + (dr - tr * g.TR)) * g.TQ + (dq - tq * g.TQ);
    key_of[i] = key;
    atomicAdd(&counts[key], 1);
  }
}

// exclusive scan of n ints in place, three passes: per-block scan, scan of block sums, add back
constexpr int kScanThreads = 1024, kScanPer = 4, kScanBlock = kScanThreads * kScanPer;
__global__ void k_scan_blocks(int* __restrict__ a, int64_t n, int* __restrict__ bsum) {
  __shared__ int ws[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer], tot = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < n) ? a[base + k] : 0;
    tot += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < kScanThreads / 32) ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) ws[lane] = w;
  }
  __syncthreads();
  int run = incl - tot + (warp > 0 ? ws[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) a[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = run;
}
__global__ void k_scan_sums(int* __restrict__ bsum, int nb) {  // one thread: nb is small
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int run = 0;
    for (int i = 0; i < nb; ++i) {
      const int v = bsum[i];
      bsum[i] = run;
      run += v;
    }
  }
}
__global__ void k_scan_add(int* __restrict__ a, int64_t n, const int* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int add = bsum[blockIdx.x];
  for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x)
    if (base + k < n) a[base + k] += add;
}

__device__ __forceinline__ double es_psi(double z, double beta) {
  if (z < -1.0 || z > 1.0) return 0.0;
  return exp(beta * (sqrt(1.0 - z * z) - 1.0));
}

// first sorted point of every (tile, base row): the scanned count at key (tile, row, column 0)
__global__ void k_row_offsets(const int* __restrict__ cnt, int64_t nr, int TQ, int* __restrict__ roff) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nr) roff[i] = cnt[i * TQ];
}

__global__ void k_tile_offsets(const int* __restrict__ cnt, int ntiles, int per_tile, int* __restrict__ toff) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= ntiles) toff[t] = cnt[(int64_t)t * per_tile];
}

__global__ void k_bin_scatter(const double* __restrict__ theta, const double* __restrict__ phi, int64_t n, BinGeom g,
                              const int* __restrict__ key_of, const int* __restrict__ offsets,
                              int* __restrict__ cursor, int32_t* __restrict__ pidx, int32_t* __restrict__ pcell,
                              double* __restrict__ pw, int4* __restrict__ prec, double beta_es) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int key = key_of[i];
    if (key < 0) continue;
    double t, u;
    point_tu(g, theta[i], phi[i], t, u);
    const int r0 = (int)ceil(t - 0.5 * g.W), q0 = (int)ceil(u - 0.5 * g.W);
    const int pos = offsets[key] + atomicAdd(&cursor[key], 1);
    const int lq = key % g.TQ, lr = (key / g.TQ) % g.TR;
    const int32_t cell = (int32_t)(lr | (lq << 16));
    if (prec) {  // FP32 form: one record
      prec[pos] = make_int4((int)i, cell, __float_as_int((float)(t - (double)r0)), __float_as_int((float)(u - (double)q0)));
      continue;
    }
    pidx[pos] = (int32_t)i;
    pcell[pos] = cell;
    if (pw) {
      for (int a = 0; a < g.W; ++a) {
        pw[(int64_t)a * n + pos] = es_psi(2.0 * (t - (double)(r0 + a)) / g.W, beta_es);
        pw[(int64_t)(g.W + a) * n + pos] = es_psi(2.0 * (u - (double)(q0 + a)) / g.W, beta_es);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
template <typename T, int W>
struct Weights;
template <int W>
struct Weights<double, W> {
  __device__ __forceinline__ static void get(const double* pw, int64_t n, int64_t pt, double* wr, double* wq) {
#pragma unroll
    for (int a = 0; a < W; ++a) {
      wr[a] = pw[(int64_t)a * n + pt];
      wq[a] = pw[(int64_t)(W + a) * n + pt];
    }
  }
};
template <int W>
struct Weights<float, W> {
  // the kernel values of the W rows and W columns from the in-cell offsets t - r0 and u - q0
  __device__ __forceinline__ static void from(float ft, float fu, float beta, float* wr, float* wq) {
    const float sc = 2.0f / W;
#pragma unroll
    for (int a = 0; a < W; ++a) {
      const float zr = (ft - (float)a) * sc, zq = (fu - (float)a) * sc;
      wr[a] = __expf(beta * (sqrtf(fmaxf(0.0f, 1.0f - zr * zr)) - 1.0f));
      wq[a] = __expf(beta * (sqrtf(fmaxf(0.0f, 1.0f - zq * zq)) - 1.0f));
    }
  }
};

// the interpolated value at one point from the shared tile: window rows lr .. lr+W-1, columns
// lq .. lq+W-1 of the tile, weights wr (rows) and wq (columns)
template <typename T, int W>
__device__ __forceinline__ typename Cx<T>::V interp_point(const typename Cx<T>::V* tile, int pitch, int cell,
                                                          const T* wr, const T* wq) {
  using V = typename Cx<T>::V;
  const int lr = cell & 0xffff, lq = cell >> 16;
  T accr = 0, acci = 0;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    const V* tp = tile + (lr + a) * pitch + lq;
    T rr = 0, ri = 0;
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const V gv = tp[b];
      rr = fma(wq[b], gv.x, rr);
      ri = fma(wq[b], gv.y, ri);
    }
    accr = fma(wr[a], rr, accr);
    acci = fma(wr[a], ri, acci);
  }
  return mk(accr, acci);
}

template <typename T, int W>
__global__ void __launch_bounds__(kInterpThreads) k_gather(const TileItem* __restrict__ items,
                                                           const int32_t* __restrict__ pidx,
                                                           const int32_t* __restrict__ pcell,
                                                           const double* __restrict__ pw,
                                                           const int4* __restrict__ prec, int64_t npts,
                                                           const typename Cx<T>::V* __restrict__ G, int nrows,
                                                           int gstride, int TR, int TQ, T beta,
                                                           typename Cx<T>::V* __restrict__ f) {
  using V = typename Cx<T>::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tile = reinterpret_cast<V*>(smraw);
  const TileItem it = items[blockIdx.x];
  const int pitch = TQ + W - 1, rows = TR + W - 1;
  const int row0 = it.tr * TR, col0 = it.tq * TQ;
  for (int e = threadIdx.x; e < rows * pitch; e += blockDim.x) {
    const int rr = e / pitch, cc = e - rr * pitch;
    const int gr = row0 + rr, gc = col0 + cc;
    tile[e] = (gr < nrows && gc < gstride) ? G[(int64_t)gr * gstride + gc] : mk((T)0, (T)0);
  }
  __syncthreads();
  // the next point's record (FP32) or cell and output index (FP64) are loaded one iteration ahead
  const int pend = it.p0 + it.np;
  int pt = it.p0 + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    int4 rn = pt < pend ? prec[pt] : make_int4(0, 0, 0, 0);
    for (; pt < pend; pt += blockDim.x) {
      const int4 rc = rn;
      if (pt + (int)blockDim.x < pend) rn = prec[pt + blockDim.x];
      T wr[W], wq[W];
      Weights<T, W>::from(__int_as_float(rc.z), __int_as_float(rc.w), beta, wr, wq);
      f[rc.x] = interp_point<T, W>(tile, pitch, rc.y, wr, wq);
    }
  } else {
    int cell_n = pt < pend ? pcell[pt] : 0, idx_n = pt < pend ? pidx[pt] : 0;
    for (; pt < pend; pt += blockDim.x) {
      const int cell = cell_n, idx = idx_n;
      if (pt + (int)blockDim.x < pend) {
        cell_n = pcell[pt + blockDim.x];
        idx_n = pidx[pt + blockDim.x];
      }
      T wr[W], wq[W];
      Weights<T, W>::get(pw, npts, pt, wr, wq);
      f[idx] = interp_point<T, W>(tile, pitch, cell, wr, wq);
    }
  }
}

// Spreading (transpose of k_gather).  Each warp owns a private copy of the tile; it spreads 32
// consecutive (cell-sorted) points at a time, one per lane.  Lanes whose points share a base cell
// take separate rounds, so within one window offset (a, b) all lanes write distinct cells; a
// __syncwarp after every offset orders the read-modify-writes of successive offsets.  The warp
// copies are summed at the end and added to the grid with one global atomic per nonzero cell.
template <typename T, int W, int NT>
__global__ void __launch_bounds__(NT) k_scatter(const TileItem* __restrict__ items, const int32_t* __restrict__ pidx,
                                                const int32_t* __restrict__ pcell, const double* __restrict__ pw,
                                                int64_t npts, const typename Cx<T>::V* __restrict__ f,
                                                typename Cx<T>::V* __restrict__ G, int nrows, int gstride, int TR,
                                                int TQ, T beta) {
  using V = typename Cx<T>::V;
  constexpr int NWARP = NT / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* tiles = reinterpret_cast<V*>(smraw);
  const TileItem it = items[blockIdx.x];
  const int pitch = TQ + W - 1, rows = TR + W - 1, cells = rows * pitch;
  const int row0 = it.tr * TR, col0 = it.tq * TQ;
  for (int e = threadIdx.x; e < NWARP * cells; e += NT) tiles[e] = mk((T)0, (T)0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  V* tw = tiles + warp * cells;
  const unsigned lt = (1u << lane) - 1u;
  // warp w takes a contiguous slice of the item's points; within it lane i takes points
  // i*ngrp .. i*ngrp + ngrp-1, so the 32 points spread at once lie in different parts of the tile and
  // rarely share a base cell (the cell-sorted order would put equal cells side by side)
  const int per_w = (it.np + NWARP - 1) / NWARP;
  const int w0 = it.p0 + warp * per_w;
  const int wn = max(0, min(per_w, it.p0 + it.np - w0));
  const int ngrp = (wn + 31) >> 5;
  for (int gi = 0; gi < ngrp; ++gi) {
    const int k = lane * ngrp + gi;
    const int pt = w0 + k;
    const bool valid = k < wn;
    int lr = 0, lq = 0, key = -1 - lane;
    T wr[W], wq[W];
    V fv = mk((T)0, (T)0);
    if (valid) {
      const int cell = pcell[pt];
      lr = cell & 0xffff;
      lq = cell >> 16;
      key = lr * pitch + lq;
      Weights<T, W>::get(pw, npts, pt, wr, wq);
      fv = f[pidx[pt]];
    } else {
#pragma unroll
      for (int a = 0; a < W; ++a) wr[a] = wq[a] = (T)0;
    }
    const unsigned same = __match_any_sync(0xffffffffu, key);
    const unsigned rank = __popc(same & lt);
    const unsigned rounds = __reduce_max_sync(0xffffffffu, rank) + 1u;
    for (unsigned rd = 0; rd < rounds; ++rd) {
      const bool on = valid && rank == rd;
#pragma unroll
      for (int a = 0; a < W; ++a) {
        const T vr = wr[a] * fv.x, vi = wr[a] * fv.y;
        V* tp = tw + (lr + a) * pitch + lq;
#pragma unroll
        for (int b = 0; b < W; ++b) {
          if (on) {
            V x = tp[b];
            x.x = fma(wq[b], vr, x.x);
            x.y = fma(wq[b], vi, x.y);
            tp[b] = x;
          }
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < cells; e += NT) {
    T vr = 0, vi = 0;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
      vr += tiles[w * cells + e].x;
      vi += tiles[w * cells + e].y;
    }
    if (vr == (T)0 && vi == (T)0) continue;
    const int rr = e / pitch, cc = e - rr * pitch;
    const int gr = row0 + rr, gc = col0 + cc;
    if (gr < nrows && gc < gstride) {
      T* gp = reinterpret_cast<T*>(G + (int64_t)gr * gstride + gc);
      atomicAdd(gp, vr);
      atomicAdd(gp + 1, vi);
    }
  }
}

// Spreading in the FP32 form, one warp per tile of 32 base rows x 16 base columns (the plan's tile
// shape in that form).  Lane i takes the points whose window starts on the tile's base row i, in
// their sorted (column) order, one point per step.  Within one row a of the windows the 32 lanes
// update 32 different grid rows (i + a), so no two lanes touch the same cell and each lane issues
// its W loads, multiply-adds and stores of that row back to back; a __syncwarp after each window
// row orders them against the next row, which the neighbouring lane updated.  The warp's private
// tile is stored column-major with a column pitch P of 48 cells (a multiple of 16 eight-byte banks),
// so a warp access to (row i + a, column q_i + b) hits bank (i + a) mod 16 in each half-warp: no
// bank conflicts whatever the lanes' columns.  The tile is then added to the grid with one vector
// atomic per nonzero cell.
constexpr int kRowTR = 32, kRowTQ = 16, kRowP = 48, kRowWarps = 8;

__device__ __forceinline__ void red_add_v2(float2* addr, float2 v) {
  asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(v.x), "f"(v.y) : "memory");
}

template <int W>
__global__ void __launch_bounds__(kRowWarps * 32) k_scatter_rows(const int* __restrict__ roff, int ntiles, int ntq,
                                                                 const int4* __restrict__ prec,
                                                                 const float2* __restrict__ f, float2* __restrict__ G,
                                                                 int nrows, int gstride, float beta) {
  static_assert(kRowTR + W - 1 <= kRowP, "window rows exceed the column pitch");
  constexpr int COLS = kRowTQ + W - 1, ROWS = kRowTR + W - 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * kRowWarps + warp;
  if (t >= ntiles) return;
  const int s0 = roff[t * kRowTR + lane], s1 = roff[t * kRowTR + lane + 1];
  int cnt = s1 - s0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, o));
  if (cnt == 0) return;  // no points in the tile
  float2* tw = reinterpret_cast<float2*>(smraw) + warp * COLS * kRowP;
  // per-point inputs loaded ahead of their use: the point's 16-byte record (index, cell, offsets)
  // two steps ahead, its value (a read at the caller's point order, so a random one) one step
  // ahead, so that no step waits on a dependent pair of loads
  const float2 z = make_float2(0.f, 0.f);
  const int4 z4 = make_int4(0, 0, 0, 0);
  int4 rec_n = z4, rec_nn = z4;
  float2 fv_n = z;
  if (s0 < s1) {
    rec_n = prec[s0];
    fv_n = f[rec_n.x];
  }
  if (s0 + 1 < s1) rec_nn = prec[s0 + 1];
  for (int e = lane; e < COLS * kRowP; e += 32) tw[e] = z;
  __syncwarp();
  for (int k = 0; k < cnt; ++k) {
    const int pt = s0 + k;
    const bool on = pt < s1;
    const int4 rc = rec_n;
    const float2 fv = fv_n;
    if (pt + 1 < s1) {
      rec_n = rec_nn;
      fv_n = f[rec_nn.x];
    }
    if (pt + 2 < s1) rec_nn = prec[pt + 2];
    int lq = 0;
    float wr[W], wq[W];
    if (on) {
      lq = rc.y >> 16;
      Weights<float, W>::from(__int_as_float(rc.z), __int_as_float(rc.w), beta, wr, wq);
    }
    float2* col = tw + lq * kRowP + lane;
#pragma unroll
    for (int a = 0; a < W; ++a) {
      if (on) {
        const float vr = wr[a] * fv.x, vi = wr[a] * fv.y;
        float2 x[W];
#pragma unroll
        for (int b = 0; b < W; ++b) x[b] = col[b * kRowP + a];
#pragma unroll
        for (int b = 0; b < W; ++b) {
          x[b].x = fmaf(wq[b], vr, x[b].x);
          x[b].y = fmaf(wq[b], vi, x[b].y);
        }
#pragma unroll
        for (int b = 0; b < W; ++b) col[b * kRowP + a] = x[b];
      }
      __syncwarp();
    }
  }
  // add the tile to the grid: lanes walk the rows of one column at a time (conflict-free reads)
  const int tr = t / ntq, tq = t - tr * ntq;
  const int row0 = tr * kRowTR, col0 = tq * kRowTQ;
  for (int c = 0; c < COLS; ++c) {
    const int gc = col0 + c;
    for (int r = lane; r < ROWS; r += 32) {
      const float2 v = tw[c * kRowP + r];
      const int gr = row0 + r;
      if ((v.x != 0.f || v.y != 0.f) && gr < nrows && gc < gstride) red_add_v2(G + (int64_t)gr * gstride + gc, v);
    }
  }
}

template <typename T, int W>
void run_gather(Plan& p, void* f, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const size_t smem = (size_t)(p.TR + W - 1) * (p.TQ + W - 1) * sizeof(V);
  allow_dynamic_smem((const void*)k_gather<T, W>, smem);
  k_gather<T, W><<<p.ntitems, kInterpThreads, smem, st>>>(p.d_titems, p.d_pidx, p.d_pcell, (const double*)p.d_pw,
                                                          p.d_prec, p.npts, (const V*)p.d_G, p.nrows, p.gstride,
                                                          p.TR, p.TQ, (T)p.beta_es, (V*)f);
}
template <typename T, int W>
void run_scatter(Plan& p, const void* f, cudaStream_t st) {
  using V = typename Cx<T>::V;
  if constexpr (sizeof(T) == 4) {  // the FP32 form's tiles are 32 x 16 with per-row point ranges
    const int ntiles = p.ntr * p.ntq;
    const size_t smem = (size_t)kRowWarps * (kRowTQ + W - 1) * kRowP * sizeof(float2);
    allow_dynamic_smem((const void*)k_scatter_rows<W>, smem);
    k_scatter_rows<W><<<(ntiles + kRowWarps - 1) / kRowWarps, kRowWarps * 32, smem, st>>>(
        p.d_roff, ntiles, p.ntq, p.d_prec, (const float2*)f, (float2*)p.d_G, p.nrows, p.gstride, (float)p.beta_es);
  } else {  // FP64: the generic tile kernel with a private tile per warp
    constexpr int NT = 128;
    const size_t smem = (size_t)(NT / 32) * (p.TR + W - 1) * (p.TQ + W - 1) * sizeof(V);
    allow_dynamic_smem((const void*)k_scatter<T, W, NT>, smem);
    k_scatter<T, W, NT><<<p.ntitems, NT, smem, st>>>(p.d_titems, p.d_pidx, p.d_pcell, (const double*)p.d_pw, p.npts,
                                                     (const V*)f, (V*)p.d_G, p.nrows, p.gstride, p.TR, p.TQ,
                                                     (T)p.beta_es);
  }
}

template <typename T, bool GATHER>
void dispatch_w(Plan& p, void* f, cudaStream_t st) {
#define PSHT_W_CASE(w)                         \
  case w:                                      \
    if (GATHER) run_gather<T, w>(p, f, st);    \
    else run_scatter<T, w>(p, f, st);          \
    break;
  if (sizeof(T) == 8) {
    switch (p.W) {
      PSHT_W_CASE(2) PSHT_W_CASE(3) PSHT_W_CASE(4) PSHT_W_CASE(5) PSHT_W_CASE(6) PSHT_W_CASE(7) PSHT_W_CASE(8)
      PSHT_W_CASE(9) PSHT_W_CASE(10) PSHT_W_CASE(11) PSHT_W_CASE(12) PSHT_W_CASE(13) PSHT_W_CASE(14)
      PSHT_W_CASE(15) PSHT_W_CASE(16)
      default: throw Error{PSHT_ENOTSUP, "kernel width outside 2..16"};
    }
  } else {
    switch (p.W) {
      PSHT_W_CASE(2) PSHT_W_CASE(3) PSHT_W_CASE(4) PSHT_W_CASE(5) PSHT_W_CASE(6) PSHT_W_CASE(7) PSHT_W_CASE(8)
      default: throw Error{PSHT_ENOTSUP, "FP32 form supports kernel widths 2..8 (eps >= 1e-7)"};
    }
  }
#undef PSHT_W_CASE
}

}  // namespace

void reduce_points(const double* theta, const double* phi, int64_t npts, double out[3], cudaStream_t st) {
  unsigned long long* d = nullptr;
  PSHT_CUDA_TRY(cudaMallocAsync((void**)&d, 3 * sizeof(unsigned long long), st));
  PSHT_CUDA_TRY(cudaMemsetAsync(d, 0, 3 * sizeof(unsigned long long), st));
  if (npts > 0) {
    const int nbl = (int)std::min<int64_t>((npts + kBinThreads - 1) / kBinThreads, 152 * 16);
    k_reduce<<<nbl, kBinThreads, 0, st>>>(theta, phi, npts, d);
    PSHT_CUDA_TRY(cudaGetLastError());
  }
  unsigned long long h[3];
  PSHT_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
  PSHT_CUDA_TRY(cudaStreamSynchronize(st));
  PSHT_CUDA_TRY(cudaFreeAsync(d, st));
  memcpy(&out[0], &h[0], sizeof(double));
  memcpy(&out[1], &h[1], sizeof(double));
  out[2] = (double)h[2];
}

void bin_points(Plan& p, const double* theta, const double* phi, cudaStream_t st) {
  const int64_t n = p.npts;
  BinGeom g;
  g.pole = p.pole;
  g.theta_max = p.theta_max;
  g.nTheta = p.nTheta;
  g.nphi = p.nphi;
  g.W = p.W;
  g.r_lo = p.r_lo;
  g.padq = p.padq;
  g.TR = p.TR;
  g.TQ = p.TQ;
  g.ntr = p.ntr;
  g.ntq = p.ntq;
  const int ntiles = p.ntr * p.ntq;
  const int64_t nkeys = (int64_t)ntiles * p.TR * p.TQ;
  PSHT_REQUIRE(nkeys < ((int64_t)1 << 31), PSHT_ENOTSUP, "grid too large for 32-bit point binning keys");
  const int64_t nsb = (nkeys + 1 + kScanBlock - 1) / kScanBlock;  // blocks of the scan over nkeys + 1 entries
  int *d_key = nullptr, *d_cnt = nullptr, *d_cur = nullptr, *d_bs = nullptr, *d_toff = nullptr;
  PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_key, sizeof(int) * std::max<int64_t>(n, 1), st));
  PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_cnt, sizeof(int) * (nkeys + 1), st));
  PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_cur, sizeof(int) * nkeys, st));
  PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_bs, sizeof(int) * std::max<int64_t>(nsb, 1), st));
  PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_toff, sizeof(int) * (ntiles + 1), st));
  PSHT_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(int) * (nkeys + 1), st));
  const int nbl = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBinThreads - 1) / kBinThreads, 152 * 32));
  if (n > 0) k_bin_count<<<nbl, kBinThreads, 0, st>>>(theta, phi, n, g, d_key, d_cnt);
  PSHT_CUDA_TRY(cudaGetLastError());
  // counting sort: exclusive scan of the per-key counts (entry nkeys becomes the total)
  const int nb = (int)nsb;
  k_scan_blocks<<<nb, kScanThreads, 0, st>>>(d_cnt, nkeys + 1, d_bs);
  k_scan_sums<<<1, 32, 0, st>>>(d_bs, nb);
  k_scan_add<<<nb, 256, 0, st>>>(d_cnt, nkeys + 1, d_bs);
  PSHT_CUDA_TRY(cudaGetLastError());
  // tile boundaries on the host: offsets of each tile's first key
  std::vector<int> toff(ntiles + 1);
  k_tile_offsets<<<(ntiles + 1 + 255) / 256, 256, 0, st>>>(d_cnt, ntiles, p.TR * p.TQ, d_toff);
  PSHT_CUDA_TRY(cudaGetLastError());
  PSHT_CUDA_TRY(cudaMemcpyAsync(toff.data(), d_toff, sizeof(int) * (ntiles + 1), cudaMemcpyDeviceToHost, st));
  PSHT_CUDA_TRY(cudaStreamSynchronize(st));
  PSHT_REQUIRE(toff[ntiles] == n, PSHT_EINVAL, "a point falls outside the planned grid rows (theta* inconsistent)");
  // tile work items, dense tiles split so that no CTA holds more than kMaxPts points
  const int kMaxPts = 2048;
  std::vector<TileItem> items;
  for (int t = 0; t < ntiles; ++t) {
    const int c = toff[t + 1] - toff[t];
    for (int b = 0; b < c; b += kMaxPts) {
      TileItem it;
      it.tr = t / p.ntq;
      it.tq = t % p.ntq;
      it.p0 = toff[t] + b;
      it.np = std::min(kMaxPts, c - b);
      items.push_back(it);
    }
  }
  p.ntitems = (int)items.size();
  if (p.ntitems > 0) {
    PSHT_CUDA_TRY(cudaMalloc((void**)&p.d_titems, sizeof(TileItem) * items.size()));
    p.allocs.push_back(p.d_titems);
    p.bytes += sizeof(TileItem) * items.size();
    PSHT_CUDA_TRY(cudaMemcpyAsync(p.d_titems, items.data(), sizeof(TileItem) * items.size(), cudaMemcpyHostToDevice, st));
  }
  if (p.prec == 32) {  // per (tile, base row) first sorted point, for the FP32 spreading kernel
    PSHT_REQUIRE(p.TR == kRowTR && p.TQ == kRowTQ, PSHT_ECUDA, "internal: FP32 tile shape");
    const int64_t nr = (int64_t)ntiles * p.TR + 1;
    PSHT_CUDA_TRY(cudaMalloc((void**)&p.d_roff, sizeof(int) * nr));
    p.allocs.push_back(p.d_roff);
    p.bytes += sizeof(int) * nr;
    k_row_offsets<<<(int)((nr + 255) / 256), 256, 0, st>>>(d_cnt, nr, p.TQ, p.d_roff);
    PSHT_CUDA_TRY(cudaGetLastError());
  }
  PSHT_CUDA_TRY(cudaMemsetAsync(d_cur, 0, sizeof(int) * nkeys, st));
  if (n > 0)
    k_bin_scatter<<<nbl, kBinThreads, 0, st>>>(theta, phi, n, g, d_key, d_cnt, d_cur, p.d_pidx, p.d_pcell,
                                               (double*)p.d_pw, p.d_prec, p.beta_es);
  PSHT_CUDA_TRY(cudaGetLastError());
  PSHT_CUDA_TRY(cudaFreeAsync(d_key, st));
  PSHT_CUDA_TRY(cudaFreeAsync(d_cnt, st));
  PSHT_CUDA_TRY(cudaFreeAsync(d_cur, st));
  PSHT_CUDA_TRY(cudaFreeAsync(d_bs, st));
  PSHT_CUDA_TRY(cudaFreeAsync(d_toff, st));
  PSHT_CUDA_TRY(cudaStreamSynchronize(st));
}

void launch_gather(Plan& p, void* f, cudaStream_t st) {
  if (p.ntitems == 0) return;
  if (p.prec == 64) dispatch_w<double, true>(p, f, st);
  else dispatch_w<float, true>(p, f, st);
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_scatter(Plan& p, const void* f, cudaStream_t st) {
  if (p.ntitems == 0) return;
  if (p.prec == 64) dispatch_w<double, false>(p, const_cast<void*>(f), st);
  else dispatch_w<float, false>(p, const_cast<void*>(f), st);
  PSHT_CUDA_TRY(cudaGetLastError());
}

}  // namespace psht
