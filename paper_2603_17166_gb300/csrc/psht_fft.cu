// FFT stages between the ring coefficients and the oversampled grid.
//
// Theta stage (per phi-order column m, Sec. I.A-B and Sec. II steps 3-4):
//   h_k = w_k F_k[m] (k <= L),  h_k = (-1)^(s+m) w_{2L-k} F_{2L-k}[m] (L < k < 2L)     (pole-crossing rule)
//   H[n] = sum_k h_k e^{-i pi n k/L},  b[n] = H[n] sT(n) sP(m) for |n| <= L-1  (ES deconvolution)
//   C[r] = sum_n b[n] e^{+2 pi i n r/nTheta} for the kept rows r in [r_lo, r_lo + nrows)
// Phi stage (per kept row):  G[r, q] = sum_{|m|<=M} C[r, m] e^{+2 pi i m q/nphi}, stored with a
// wrapped halo of padq columns on both sides.
// The adjoint kernels apply the exact transposes in reverse order.
// Every transform runs in place in shared memory (psht_common.cuh), one CTA per column or row.
#include <cuda_runtime.h>

#include <algorithm>

#include "psht_common.cuh"

namespace psht {

namespace {

constexpr int kFftThreads = 512;
// longest transforms held in one CTA's shared memory (227 KiB) with the padded layout (PadBuf)
constexpr int kMaxLenF64 = 14000;  // complex128
constexpr int kMaxLenF32 = 28000;  // complex64
// |n| <= L-1 values held per thread while the buffer is re-laid out (2L <= max length / 2)
// threads of the Theta kernels per launch mode (see k_theta_syn)
__host__ __device__ constexpr int theta_threads(int mode) { return mode == 1 ? 256 : kFftThreads; }

template <typename T>
struct QPer {
  static constexpr int v = ((sizeof(T) == 8 ? kMaxLenF64 : kMaxLenF32) / 2 + kFftThreads - 1) / kFftThreads;
};

// MODE 1: one CTA of 256 threads per column, the transform in shared memory and the |n| <= L-1
// values staged behind it (4L + 2L elements).  MODE 0 (when 6L elements exceed shared memory): 512
// threads, the 4L-element transform in shared memory and those values held in registers between
// the two transforms.  MODE 2 (lengths beyond shared memory): gridDim.x CTAs loop over the columns,
// each with its own 6L-element slice of a global scratch array, which the L2 cache holds.
template <typename T, int MODE>
__global__ void __launch_bounds__(theta_threads(MODE)) k_theta_syn(const typename Cx<T>::V* __restrict__ F, int Lpad,
                                                           const T* __restrict__ w, int nring,
                                                           const int2* __restrict__ mrange, int mstride, int s, int L,
                                                           const T* __restrict__ sT, const T* __restrict__ sP, int M,
                                                           FftDev f2L, const typename Cx<T>::V* __restrict__ tw2L,
                                                           const int* __restrict__ perm2L, FftDev f4L,
                                                           const typename Cx<T>::V* __restrict__ tw4L,
                                                           const int* __restrict__ perm4L, int r_lo, int nrows,
                                                           typename Cx<T>::V* __restrict__ X, int ncols,
                                                           typename Cx<T>::V* __restrict__ scratch) {
  using V = typename Cx<T>::V;
  constexpr bool GM = MODE == 2;   // global buffers, columns looped over a persistent grid
  constexpr bool STG = MODE != 0;  // |n| <= L-1 values staged behind the transform, not in registers
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N2 = 2 * L, N4 = 4 * L;
  V* const raw = GM ? scratch + (int64_t)blockIdx.x * (padded_len(N4) + N2) : reinterpret_cast<V*>(smraw);
  const PadBuf<V> buf{raw};
  auto body = [&](const int mi) {
  const int m = col_m(mi), am = m < 0 ? -m : m;
  const T sigma = ((s + am) & 1) ? (T)-1 : (T)1;
  const int2 rr = mrange[am], rr1 = mrange[mstride + am];  // active rings: direct part, reflected part
  const V* Fc = F + (int64_t)mi * Lpad;
  for (int k = threadIdx.x; k < N2; k += blockDim.x) {
    int j = k;
    T sg = (T)1;
    if (k > L) {
      j = N2 - k;
      sg = sigma;
    }
    V v = mk((T)0, (T)0);
    if (j < nring && ((j >= rr.x && j < rr.y) || (j >= rr1.x && j < rr1.y))) v = cscale(Fc[j], sg * w[j]);
    buf[k] = v;
  }
  __syncthreads();
  fft_dif<false>(buf, f2L, tw2L);
  // collect b[n] = H[n] sT(n) sP(m), |n| <= L-1, then lay them out for the inverse DIT of length 4L
  const T sp = sP[m + M];
  if constexpr (STG) {
    V* stg = raw + padded_len(N4);
    for (int i = threadIdx.x; i < N2 - 1; i += blockDim.x) {
      const int n = i - (L - 1);
      stg[i] = cscale(buf[perm2L[n < 0 ? n + N2 : n]], sT[i] * sp);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N4; k += blockDim.x) buf[k] = mk((T)0, (T)0);
    __syncthreads();
    for (int i = threadIdx.x; i < N2 - 1; i += blockDim.x) {
      const int n = i - (L - 1);
      buf[perm4L[n < 0 ? n + N4 : n]] = stg[i];
    }
  } else {
    constexpr int kQ = QPer<T>::v;
    V hv[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int i = threadIdx.x + q * blockDim.x;
      if (i < N2 - 1) {
        const int n = i - (L - 1);
        hv[q] = cscale(buf[perm2L[n < 0 ? n + N2 : n]], sT[i] * sp);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N4; k += blockDim.x) buf[k] = mk((T)0, (T)0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int i = threadIdx.x + q * blockDim.x;
      if (i < N2 - 1) {
        const int n = i - (L - 1);
        buf[perm4L[n < 0 ? n + N4 : n]] = hv[q];
      }
    }
  }
  __syncthreads();
  fft_dit<true>(buf, f4L, tw4L);
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    int r = (r_lo + i) % N4;
    if (r < 0) r += N4;
    X[(int64_t)i * ncols + mi] = buf[r];
  }
  __syncthreads();  // buf is reused by the next column
  };
  if constexpr (GM) {
    for (int mi = blockIdx.x; mi < ncols; mi += gridDim.x) body(mi);
  } else {
    body(blockIdx.x);
  }
}

// GM as for k_theta_syn: rows looped over gridDim.x CTAs, each with an nphi-element scratch slice
template <typename T, bool GM>
__global__ void __launch_bounds__(kFftThreads) k_phi_syn(const typename Cx<T>::V* __restrict__ X, int ncols,
                                                         FftDev fP, const typename Cx<T>::V* __restrict__ twP,
                                                         const int* __restrict__ permP, int padq, int gstride,
                                                         typename Cx<T>::V* __restrict__ G, int nrows,
                                                         typename Cx<T>::V* __restrict__ scratch) {
  using V = typename Cx<T>::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nphi = fP.n;
  const PadBuf<V> buf{GM ? scratch + (int64_t)blockIdx.x * padded_len(nphi) : reinterpret_cast<V*>(smraw)};
  auto body = [&](const int row) {
  for (int k = threadIdx.x; k < nphi; k += blockDim.x) buf[k] = mk((T)0, (T)0);
  __syncthreads();
  const V* Xr = X + (int64_t)row * ncols;
  for (int mi = threadIdx.x; mi < ncols; mi += blockDim.x) {
    const int m = col_m(mi);
    buf[permP[m < 0 ? m + nphi : m]] = Xr[mi];
  }
  __syncthreads();
  fft_dit<true>(buf, fP, twP);
  V* Gr = G + (int64_t)row * gstride;
  const int nq = nphi + 2 * padq;
  if (nphi >= 2 * padq) {  // each halo wraps once
#pragma unroll 4
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      int src = q - padq;
      src += src < 0 ? nphi : (src >= nphi ? -nphi : 0);
      Gr[q] = buf[src];
    }
  } else {
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      int src = (q - padq) % nphi;  // the halo may wrap more than once when nphi < padq
      if (src < 0) src += nphi;
      Gr[q] = buf[src];
    }
  }
  for (int q = nq + threadIdx.x; q < gstride; q += blockDim.x) Gr[q] = mk((T)0, (T)0);
  __syncthreads();  // buf is reused by the next row
  };
  if constexpr (GM) {
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) body(row);
  } else {
    body(blockIdx.x);
  }
}

template <typename T, bool GM>
__global__ void __launch_bounds__(kFftThreads) k_phi_adj(const typename Cx<T>::V* __restrict__ G, int gstride,
                                                         int padq, FftDev fP, const typename Cx<T>::V* __restrict__ twP,
                                                         const int* __restrict__ permP,
                                                         typename Cx<T>::V* __restrict__ X, int ncols, int nrows,
                                                         typename Cx<T>::V* __restrict__ scratch) {
  using V = typename Cx<T>::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nphi = fP.n;
  const PadBuf<V> buf{GM ? scratch + (int64_t)blockIdx.x * padded_len(nphi) : reinterpret_cast<V*>(smraw)};
  auto body = [&](const int row) {
  const V* Gr = G + (int64_t)row * gstride;
  // fold every stored column qs (true column qs - padq) onto q = (qs - padq) mod nphi
  const int nq = nphi + 2 * padq;
  if (nphi >= 2 * padq) {  // each halo wraps once: a main load plus at most one halo load per q
#pragma unroll 4
    for (int q = threadIdx.x; q < nphi; q += blockDim.x) {
      V v = Gr[q + padq];
      if (q < padq) v = cadd(v, Gr[q + padq + nphi]);
      if (q >= nphi - padq) v = cadd(v, Gr[q + padq - nphi]);
      buf[q] = v;
    }
  } else {
    for (int q = threadIdx.x; q < nphi; q += blockDim.x) {
      V v = mk((T)0, (T)0);
      for (int qs = (q + padq) % nphi; qs < nq; qs += nphi) v = cadd(v, Gr[qs]);
      buf[q] = v;
    }
  }
  __syncthreads();
  fft_dif<false>(buf, fP, twP);
  V* Xr = X + (int64_t)row * ncols;
  for (int mi = threadIdx.x; mi < ncols; mi += blockDim.x) {
    const int m = col_m(mi);
    Xr[mi] = buf[permP[m < 0 ? m + nphi : m]];
  }
  __syncthreads();  // buf is reused by the next row
  };
  if constexpr (GM) {
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) body(row);
  } else {
    body(blockIdx.x);
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(theta_threads(MODE)) k_theta_adj(const typename Cx<T>::V* __restrict__ X, int ncols,
                                                           int r_lo, int nrows, const T* __restrict__ w, int nring,
                                                           int s, int L, const T* __restrict__ sT,
                                                           const T* __restrict__ sP, int M, FftDev f2L,
                                                           const typename Cx<T>::V* __restrict__ tw2L,
                                                           const int* __restrict__ perm2L, FftDev f4L,
                                                           const typename Cx<T>::V* __restrict__ tw4L,
                                                           const int* __restrict__ perm4L,
                                                           typename Cx<T>::V* __restrict__ Ft, int Lpad,
                                                           typename Cx<T>::V* __restrict__ scratch) {
  using V = typename Cx<T>::V;
  constexpr bool GM = MODE == 2;   // global buffers, columns looped over a persistent grid
  constexpr bool STG = MODE != 0;  // |n| <= L-1 values staged behind the transform, not in registers
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N2 = 2 * L, N4 = 4 * L;
  V* const raw = GM ? scratch + (int64_t)blockIdx.x * (padded_len(N4) + N2) : reinterpret_cast<V*>(smraw);
  const PadBuf<V> buf{raw};
  auto body = [&](const int mi) {
  const int m = col_m(mi), am = m < 0 ? -m : m;
  const T sigma = ((s + am) & 1) ? (T)-1 : (T)1;
  // transpose of the row read-out: row r lands on r mod 4L, summing rows that coincide
  for (int k = threadIdx.x; k < N4; k += blockDim.x) {
    int i0 = (k - r_lo) % N4;  // first row index i >= 0 with r_lo + i = k (mod 4L)
    if (i0 < 0) i0 += N4;
    V v = mk((T)0, (T)0);
    for (int i = i0; i < nrows; i += N4) v = cadd(v, X[(int64_t)i * ncols + mi]);
    buf[k] = v;
  }
  __syncthreads();
  fft_dif<false>(buf, f4L, tw4L);
  const T sp = sP[m + M];
  if constexpr (STG) {
    V* stg = raw + padded_len(N4);
    for (int i = threadIdx.x; i < N2 - 1; i += blockDim.x) {
      const int n = i - (L - 1);
      stg[i] = cscale(buf[perm4L[n < 0 ? n + N4 : n]], sT[i] * sp);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N2; k += blockDim.x) buf[k] = mk((T)0, (T)0);
    __syncthreads();
    for (int i = threadIdx.x; i < N2 - 1; i += blockDim.x) {
      const int n = i - (L - 1);
      buf[perm2L[n < 0 ? n + N2 : n]] = stg[i];
    }
  } else {
    constexpr int kQ = QPer<T>::v;
    V hv[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int i = threadIdx.x + q * blockDim.x;
      if (i < N2 - 1) {
        const int n = i - (L - 1);
        hv[q] = cscale(buf[perm4L[n < 0 ? n + N4 : n]], sT[i] * sp);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N2; k += blockDim.x) buf[k] = mk((T)0, (T)0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int i = threadIdx.x + q * blockDim.x;
      if (i < N2 - 1) {
        const int n = i - (L - 1);
        buf[perm2L[n < 0 ? n + N2 : n]] = hv[q];
      }
    }
  }
  __syncthreads();
  fft_dit<true>(buf, f2L, tw2L);
  V* Fc = Ft + (int64_t)mi * Lpad;
  for (int j = threadIdx.x; j < nring; j += blockDim.x) {
    V v = buf[j];
    if (j >= 1 && j <= L - 1) v = cadd(v, cscale(buf[N2 - j], sigma));
    Fc[j] = cscale(v, w[j]);
  }
  __syncthreads();  // buf is reused by the next column
  };
  if constexpr (GM) {
    for (int mi = blockIdx.x; mi < ncols; mi += gridDim.x) body(mi);
  } else {
    body(blockIdx.x);
  }
}

// F[mi][j] (column layout, active rings only) -> out[j][m + M], zero outside the active range
template <typename T>
__global__ void k_export_rings(const typename Cx<T>::V* __restrict__ F, int Lpad, const int2* __restrict__ mrange,
                               int mstride, int nring, int M, typename Cx<T>::V* __restrict__ out) {
  using V = typename Cx<T>::V;
  const int ncols = 2 * M + 1;
  const int64_t tot = (int64_t)nring * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / ncols);
    const int m = (int)(e % ncols) - M;
    const int am = m < 0 ? -m : m;
    const int2 rr = mrange[am], rr1 = mrange[mstride + am];
    V v = mk((T)0, (T)0);
    if ((j >= rr.x && j < rr.y) || (j >= rr1.x && j < rr1.y)) v = F[(int64_t)col_of(m) * Lpad + j];
    out[e] = v;
  }
}


}  // namespace

int max_fft_len(int prec) { return prec == 64 ? kMaxLenF64 : kMaxLenF32; }

// Lengths above one CTA's shared memory run in global-buffer mode on a persistent grid.
namespace {
constexpr int kGmCtas = 152 * 4;
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory one CTA may use
bool theta_gm(const Plan& p) { return 4 * p.L > max_fft_len(p.prec); }
bool phi_gm(const Plan& p) { return p.nphi > max_fft_len(p.prec); }
}  // namespace

size_t fft_scratch_elems(const Plan& p) {
  size_t e = 0;
  if (theta_gm(p)) e = std::max(e, (size_t)std::min(p.ncols, kGmCtas) * (padded_len(4 * p.L) + 2 * p.L));
  if (phi_gm(p)) e = std::max(e, (size_t)std::min(p.nrows, kGmCtas) * padded_len(p.nphi));
  return e;
}

// launch mode of the Theta kernels: 2 global buffers, 1 shared memory with staging, 0 registers
template <typename T>
int theta_mode(const Plan& p) {
  if (theta_gm(p)) return 2;
  return (size_t)(padded_len(4 * p.L) + 2 * p.L) * sizeof(typename Cx<T>::V) <= kMaxSmem ? 1 : 0;
}
// shared memory of the Theta kernels: the padded 4L buffer, plus the 2L staging in mode 1
template <typename T>
size_t theta_smem(const Plan& p, int mode) {
  if (mode == 2) return 0;
  return (size_t)(padded_len(4 * p.L) + (mode == 1 ? 2 * p.L : 0)) * sizeof(typename Cx<T>::V);
}

template <typename T>
void theta_syn_t(Plan& p, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const int mode = theta_mode<T>(p);
  const size_t smem = theta_smem<T>(p, mode);
  const auto fn = mode == 2 ? k_theta_syn<T, 2> : (mode == 1 ? k_theta_syn<T, 1> : k_theta_syn<T, 0>);
  if (mode != 2) allow_dynamic_smem((const void*)fn, smem);
  fn<<<mode == 2 ? std::min(p.ncols, kGmCtas) : p.ncols, theta_threads(mode), smem, st>>>(
      (const V*)p.d_F, p.Lpad, (const T*)p.d_w, p.nring, p.d_mrange, p.lmax + 1, p.spin, p.L, (const T*)p.d_sT,
      (const T*)p.d_sP, p.M, p.f2L, (const V*)p.d_tw2L, p.d_perm2L, p.f4L, (const V*)p.d_tw4L, p.d_perm4L, p.r_lo,
      p.nrows, (V*)p.d_X, p.ncols, (V*)p.d_fscratch);
  PSHT_CUDA_TRY(cudaGetLastError());
}
template <typename T>
void theta_adj_t(Plan& p, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const int mode = theta_mode<T>(p);
  const size_t smem = theta_smem<T>(p, mode);
  const auto fn = mode == 2 ? k_theta_adj<T, 2> : (mode == 1 ? k_theta_adj<T, 1> : k_theta_adj<T, 0>);
  if (mode != 2) allow_dynamic_smem((const void*)fn, smem);
  fn<<<mode == 2 ? std::min(p.ncols, kGmCtas) : p.ncols, theta_threads(mode), smem, st>>>(
      (const V*)p.d_X, p.ncols, p.r_lo, p.nrows, (const T*)p.d_w, p.nring, p.spin, p.L, (const T*)p.d_sT,
      (const T*)p.d_sP, p.M, p.f2L, (const V*)p.d_tw2L, p.d_perm2L, p.f4L, (const V*)p.d_tw4L, p.d_perm4L,
      (V*)p.d_F, p.Lpad, (V*)p.d_fscratch);
  PSHT_CUDA_TRY(cudaGetLastError());
}
template <typename T>
void phi_syn_t(Plan& p, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const bool gm = phi_gm(p);
  const size_t smem = gm ? 0 : (size_t)padded_len(p.nphi) * sizeof(V);
  const auto fn = gm ? k_phi_syn<T, true> : k_phi_syn<T, false>;
  if (!gm) allow_dynamic_smem((const void*)fn, smem);
  fn<<<gm ? std::min(p.nrows, kGmCtas) : p.nrows, kFftThreads, smem, st>>>(
      (const V*)p.d_X, p.ncols, p.fP, (const V*)p.d_twP, p.d_permP, p.padq, p.gstride, (V*)p.d_G, p.nrows,
      (V*)p.d_fscratch);
  PSHT_CUDA_TRY(cudaGetLastError());
}
template <typename T>
void phi_adj_t(Plan& p, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const bool gm = phi_gm(p);
  const size_t smem = gm ? 0 : (size_t)padded_len(p.nphi) * sizeof(V);
  const auto fn = gm ? k_phi_adj<T, true> : k_phi_adj<T, false>;
  if (!gm) allow_dynamic_smem((const void*)fn, smem);
  fn<<<gm ? std::min(p.nrows, kGmCtas) : p.nrows, kFftThreads, smem, st>>>(
      (const V*)p.d_G, p.gstride, p.padq, p.fP, (const V*)p.d_twP, p.d_permP, (V*)p.d_X, p.ncols, p.nrows,
      (V*)p.d_fscratch);
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_theta_synthesis(Plan& p, cudaStream_t st) {
  if (p.nrows == 0) return;
  if (p.prec == 64) theta_syn_t<double>(p, st);
  else theta_syn_t<float>(p, st);
}
void launch_phi_synthesis(Plan& p, cudaStream_t st) {
  if (p.nrows == 0) return;
  if (p.prec == 64) phi_syn_t<double>(p, st);
  else phi_syn_t<float>(p, st);
}
void launch_phi_adjoint(Plan& p, cudaStream_t st) {
  if (p.nrows == 0) return;
  if (p.prec == 64) phi_adj_t<double>(p, st);
  else phi_adj_t<float>(p, st);
}
void launch_theta_adjoint(Plan& p, cudaStream_t st) {
  if (p.nrows == 0) return;
  if (p.prec == 64) theta_adj_t<double>(p, st);
  else theta_adj_t<float>(p, st);
}

void launch_ring_coeffs_export(Plan& p, void* out, cudaStream_t st) {
  const int nth = 256, nbl = 152 * 8;
  if (p.prec == 64)
    k_export_rings<double><<<nbl, nth, 0, st>>>((const double2*)p.d_F, p.Lpad, p.d_mrange, p.lmax + 1, p.nring, p.M,
                                                (double2*)out);
  else
    k_export_rings<float><<<nbl, nth, 0, st>>>((const float2*)p.d_F, p.Lpad, p.d_mrange, p.lmax + 1, p.nring, p.M,
                                               (float2*)out);
  PSHT_CUDA_TRY(cudaGetLastError());
}

}  // namespace psht
