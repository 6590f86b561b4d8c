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
constexpr int kSpreadThreads = 512;  // one thread per cell of a kTileR x kTileQ output tile
constexpr int kTileR = 16, kTileQ = 32;

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

__global__ void k_tile_offsets(const int* __restrict__ cnt, int ntiles, int per_tile, int* __restrict__ toff) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= ntiles) toff[t] = cnt[(int64_t)t * per_tile];
}

__global__ void k_bin_scatter(const double* __restrict__ theta, const double* __restrict__ phi, int64_t n, BinGeom g,
                              const int* __restrict__ key_of, const int* __restrict__ offsets,
                              int* __restrict__ cursor, int32_t* __restrict__ pidx, int32_t* __restrict__ pcell,
                              double* __restrict__ pw, float* __restrict__ pfrac, double beta_es) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int key = key_of[i];
    if (key < 0) continue;
    double t, u;
    point_tu(g, theta[i], phi[i], t, u);
    const int r0 = (int)ceil(t - 0.5 * g.W), q0 = (int)ceil(u - 0.5 * g.W);
    const int pos = offsets[key] + atomicAdd(&cursor[key], 1);
    pidx[pos] = (int32_t)i;
    const int lq = key % g.TQ, lr = (key / g.TQ) % g.TR;
    pcell[pos] = (int32_t)(lr | (lq << 16));
    if (pw) {
      for (int a = 0; a < g.W; ++a) {
        pw[(int64_t)a * n + pos] = es_psi(2.0 * (t - (double)(r0 + a)) / g.W, beta_es);
        pw[(int64_t)(g.W + a) * n + pos] = es_psi(2.0 * (u - (double)(q0 + a)) / g.W, beta_es);
      }
    }
    if (pfrac) {
      pfrac[pos] = (float)(t - (double)r0);
      pfrac[n + pos] = (float)(u - (double)q0);
    }
  }
}

// ---------------------------------------------------------------------------------------------
template <typename T, int W>
struct Weights;
template <int W>
struct Weights<double, W> {
  __device__ __forceinline__ static void get(const double* pw, const float*, int64_t n, int64_t pt, double, double* wr,
                                             double* wq) {
#pragma unroll
    for (int a = 0; a < W; ++a) {
      wr[a] = pw[(int64_t)a * n + pt];
      wq[a] = pw[(int64_t)(W + a) * n + pt];
    }
  }
};
template <int W>
struct Weights<float, W> {
  __device__ __forceinline__ static void get(const double*, const float* pf, int64_t n, int64_t pt, float beta,
                                             float* wr, float* wq) {
    const float ft = pf[pt], fu = pf[n + pt];
    const float sc = 2.0f / W;
#pragma unroll
    for (int a = 0; a < W; ++a) {
      const float zr = (ft - (float)a) * sc, zq = (fu - (float)a) * sc;
      wr[a] = __expf(beta * (sqrtf(fmaxf(0.0f, 1.0f - zr * zr)) - 1.0f));
      wq[a] = __expf(beta * (sqrtf(fmaxf(0.0f, 1.0f - zq * zq)) - 1.0f));
    }
  }
};

template <typename T, int W>
__global__ void __launch_bounds__(kInterpThreads) k_gather(const TileItem* __restrict__ items,
                                                           const int32_t* __restrict__ pidx,
                                                           const int32_t* __restrict__ pcell,
                                                           const double* __restrict__ pw,
                                                           const float* __restrict__ pf, int64_t npts,
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
  for (int pt = it.p0 + threadIdx.x; pt < it.p0 + it.np; pt += blockDim.x) {
    const int cell = pcell[pt];
    const int lr = cell & 0xffff, lq = cell >> 16;
    T wr[W], wq[W];
    Weights<T, W>::get(pw, pf, npts, pt, beta, wr, wq);
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
    f[pidx[pt]] = mk(accr, acci);
  }
}

// Spreading (transpose of k_gather) in output-stationary form: one CTA per output tile of TR x TQ
// grid cells, one thread per cell.  A cell (i, q) receives f_p psi_r[i - r0] psi_q[q - q0] from every
// point whose base cell (r0, q0) lies in [i-W+1, i] x [q-W+1, q], so the CTA gathers the points of
// the base-cell region [R0-W+1, R0+TR) x [Q0-W+1, Q0+TQ), which spans at most four point tiles,
// into shared memory ordered region row by region row (per row: left tile's cells, then this
// tile's), with each point's kernel weights computed once.  Each thread then reads, for each of its
// W base rows, the contiguous run of points of the W base cells to its left.  Every grid cell is
// written exactly once: no clearing pass, no atomics, and a fixed summation order.
template <typename T, int W>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(const int* __restrict__ keyofs,
                                                           const int32_t* __restrict__ pidx,
                                                           const double* __restrict__ pw,
                                                           const float* __restrict__ pf, int64_t npts,
                                                           const typename Cx<T>::V* __restrict__ f,
                                                           typename Cx<T>::V* __restrict__ G, int nrows,
                                                           int gstride, int ntr, int ntq, T beta, int batch) {
  using V = typename Cx<T>::V;
  constexpr int TR = kTileR, TQ = kTileQ;
  constexpr int RR = TR + W - 1, CC = TQ + W - 1, NREG = RR * CC;
  static_assert(NREG <= 3 * kSpreadThreads, "region scan covers three cells per thread");
  __shared__ int cofs[NREG + 1];  // region cell -> first staged index (exclusive prefix of counts)
  __shared__ int gofs[NREG];      // region cell -> first sorted point index
  __shared__ int wsum[kSpreadThreads / 32];
  extern __shared__ __align__(16) unsigned char smraw[];
  V* fv = reinterpret_cast<V*>(smraw);                                   // [batch]
  T* wts = reinterpret_cast<T*>(smraw + sizeof(V) * batch);             // [batch][2W]: psi_r, psi_q
  unsigned char* kap = smraw + (sizeof(V) + 2 * W * sizeof(T)) * batch;  // [batch] region column
  const int tid = threadIdx.x;
  const int R0 = blockIdx.y * TR, Q0 = blockIdx.x * TQ;

  // point counts of the region's base cells, from the per-cell offsets of the binning sort
  int cnt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int c = 3 * tid + k;
    cnt[k] = 0;
    if (c < NREG) {
      const int rho = c / CC, kc = c - rho * CC;
      const int dr = R0 - (W - 1) + rho, dq = Q0 - (W - 1) + kc;
      int g0 = 0;
      if (dr >= 0 && dq >= 0) {
        const int tr = dr / TR, tq = dq / TQ;
        if (tr < ntr && tq < ntq) {
          const int64_t key = ((int64_t)(tr * ntq + tq) * TR + (dr - tr * TR)) * TQ + (dq - tq * TQ);
          g0 = keyofs[key];
          cnt[k] = keyofs[key + 1] - g0;
        }
      }
      gofs[c] = g0;
    }
  }
  // block exclusive scan of the counts (three consecutive cells per thread)
  const int lane = tid & 31, warp = tid >> 5;
  const int tot = cnt[0] + cnt[1] + cnt[2];
  int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kSpreadThreads / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kSpreadThreads / 32) wsum[lane] = w;
  }
  __syncthreads();
  int run = incl - tot + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int c = 3 * tid + k;
    if (c < NREG) cofs[c] = run;
    run += cnt[k];
  }
  if (tid == kSpreadThreads - 1) cofs[NREG] = run;
  __syncthreads();
  const int total = cofs[NREG];

  const int a = tid / TQ, b = tid - a * TQ;
  const bool inside = (R0 + a < nrows) && (Q0 + b < gstride);
  T accr = 0, acci = 0;
  for (int B0 = 0; B0 < total; B0 += batch) {
    const int B1 = min(total, B0 + batch);
    if (B0 > 0) __syncthreads();  // the previous batch is consumed
    for (int c = tid; c < NREG; c += kSpreadThreads) {
      const int s0 = cofs[c], s1 = cofs[c + 1];
      for (int sidx = max(s0, B0); sidx < min(s1, B1); ++sidx) {
        const int gi = gofs[c] + (sidx - s0);
        const int slot = sidx - B0;
        fv[slot] = f[pidx[gi]];
        Weights<T, W>::get(pw, pf, npts, gi, beta, wts + (size_t)slot * 2 * W, wts + (size_t)slot * 2 * W + W);
        kap[slot] = (unsigned char)(c % CC);
      }
    }
    __syncthreads();
    if (inside) {
#pragma unroll
      for (int d = 0; d < W; ++d) {  // base row i - d is region row a + W - 1 - d
        const int c0 = (a + W - 1 - d) * CC + b;  // base columns q-W+1 .. q are region columns b .. b+W-1
        const int lo = max(cofs[c0], B0), hi = min(cofs[c0 + W], B1);
        for (int sidx = lo; sidx < hi; ++sidx) {
          const int slot = sidx - B0;
          const int e = b + W - 1 - kap[slot];
          const T* ws = wts + (size_t)slot * 2 * W;
          const T w = ws[d] * ws[W + e];
          const V x = fv[slot];
          accr = fma(w, x.x, accr);
          acci = fma(w, x.y, acci);
        }
      }
    }
  }
  if (inside) G[(int64_t)(R0 + a) * gstride + Q0 + b] = mk(accr, acci);
}

template <typename T, int W>
void run_gather(Plan& p, void* f, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const size_t smem = (size_t)(p.TR + W - 1) * (p.TQ + W - 1) * sizeof(V);
  PSHT_CUDA_TRY(cudaFuncSetAttribute((const void*)k_gather<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  k_gather<T, W><<<p.ntitems, kInterpThreads, smem, st>>>(p.d_titems, p.d_pidx, p.d_pcell, (const double*)p.d_pw,
                                                          p.d_pfrac, p.npts, (const V*)p.d_G, p.nrows, p.gstride,
                                                          p.TR, p.TQ, (T)p.beta_es, (V*)f);
}
template <typename T, int W>
void run_scatter(Plan& p, const void* f, cudaStream_t st) {
  using V = typename Cx<T>::V;
  // staged points per batch: within 64 KB (FP32) / 96 KB (FP64) of shared memory per CTA
  const size_t per_pt = sizeof(V) + 2 * W * sizeof(T) + 1;
  const int batch = (int)(((sizeof(T) == 8 ? 96 : 64) * 1024) / per_pt) / 16 * 16;
  const size_t smem = per_pt * batch + 16;
  PSHT_CUDA_TRY(cudaFuncSetAttribute((const void*)k_spread<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  const dim3 grid((p.gstride + kTileQ - 1) / kTileQ, (p.nrows + kTileR - 1) / kTileR);
  k_spread<T, W><<<grid, kSpreadThreads, smem, st>>>(p.d_keyofs, p.d_pidx, (const double*)p.d_pw, p.d_pfrac,
                                                     p.npts, (const V*)f, (V*)p.d_G, p.nrows, p.gstride, p.ntr,
                                                     p.ntq, (T)p.beta_es, batch);
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
  // the per-key offsets stay with the plan (the spreading kernel reads them)
  PSHT_CUDA_TRY(cudaMalloc((void**)&d_cnt, sizeof(int) * (nkeys + 1)));
  p.allocs.push_back(d_cnt);
  p.bytes += sizeof(int) * (nkeys + 1);
  p.d_keyofs = d_cnt;
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
  PSHT_CUDA_TRY(cudaMemsetAsync(d_cur, 0, sizeof(int) * nkeys, st));
  if (n > 0)
    k_bin_scatter<<<nbl, kBinThreads, 0, st>>>(theta, phi, n, g, d_key, d_cnt, d_cur, p.d_pidx, p.d_pcell,
                                               (double*)p.d_pw, p.d_pfrac, p.beta_es);
  PSHT_CUDA_TRY(cudaGetLastError());
  PSHT_CUDA_TRY(cudaFreeAsync(d_key, st));
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
  PSHT_REQUIRE(p.TR == kTileR && p.TQ == kTileQ, PSHT_ECUDA, "internal: tile shape differs from the spreading kernel's");
  if (p.prec == 64) dispatch_w<double, false>(p, const_cast<void*>(f), st);
  else dispatch_w<float, false>(p, const_cast<void*>(f), st);
  PSHT_CUDA_TRY(cudaGetLastError());
}

}  // namespace psht
