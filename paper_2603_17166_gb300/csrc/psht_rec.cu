// Wigner-d recursion onto the apodised rings (synthesis, "K-REC") and its transpose
// (adjoint, "K-REC-ADJ").
//
// Per order m and ring j the two columns e1_l = N_l d^l_{m,-s}(theta_j) and e2_l = N_l d^l_{m,s}(theta_j)
// follow the textbook three-term recurrence in l (the appendix's eq. Ylm gives
// sY_lm = N_l d^l_{m,-s} e^{im phi}).  The recurrence coefficients, N_l and a per-(l, m) rescaling
// kappa_l are folded into one table so that one step is y_{l+1} = (A'_l x +- B'_l) y_l - y_{l-1},
// with e_l = kappa_l y_l (kappa_{l0} = kappa_{l0+1} = 1, kappa_{l+1} = C_l kappa_{l-1}).
// Seeds are Wigner's closed form at l0 = max(m, s), evaluated in FP64 in log2 form; values too
// small for the working precision are carried as y * 2^(-F k) and join the sums once k = 0.
//
// Synthesis (eq. syn restricted to ring j):
//   F_j[m]  = -sum_l kappa_l (g + i c)_lm y1_l,   F_j[-m] = -(-1)^s sum_l kappa_l (g* + i c*)_lm y2_l
// Adjoint (transpose, then the adjoint synthesis general projection of Sec. I):
//   ut_{l,m} = -kappa_l sum_j y1_l(j) Ft_j[m],  ut_{l,-m} = -(-1)^(m-s) kappa_l sum_j y2_l(j) Ft_j[-m]
//   g~ = (ut_lm + (-1)^m conj ut_{l,-m})/2,  c~ = (ut_lm - (-1)^m conj ut_{l,-m})/(2i)
#include <cuda_runtime.h>
#include <math.h>

#include "psht_common.cuh"

namespace psht {

namespace {

constexpr int kCH = 64;  // l values staged in shared memory per chunk

__device__ __forceinline__ int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// ---------------------------------------------------------------------------------------------
// table (A'_l, B'_l, kappa_l) for every packed (l, m); one thread per m, FP64 throughout.
template <typename T>
__global__ void k_rec_table(int lmax, int s, T* __restrict__ tA, T* __restrict__ tB, T* __restrict__ tK) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > lmax) return;
  const int l0 = max(m, s);
  const int64_t base = alm_base(lmax, m);
  for (int l = m; l < l0 && l <= lmax; ++l) {
    tA[base + l] = 0;
    tB[base + l] = 0;
    tK[base + l] = 0;
  }
  const double m2 = (double)m * m, s2 = (double)s * s;
  double kprev = 1.0, kcur = 1.0;
  for (int l = l0; l <= lmax; ++l) {
    const double lp1 = l + 1.0;
    const double a = lp1 * (2.0 * l + 1.0) / sqrt((lp1 * lp1 - m2) * (lp1 * lp1 - s2));
    const double Ac = sqrt((2.0 * l + 3.0) / (2.0 * l + 1.0)) * a;
    const double Bt = (l == 0) ? 0.0 : Ac * (double)m * (double)s / ((double)l * lp1);
    double knext;
    if (l == l0) {
      knext = 1.0;
    } else {
      const double c = sqrt(((double)l * l - m2) * ((double)l * l - s2)) / ((double)l * (2.0 * l + 1.0));
      const double C = sqrt((2.0 * l + 3.0) / (2.0 * l - 1.0)) * a * c;
      knext = C * kprev;
    }
    tK[base + l] = (T)kcur;
    tA[base + l] = (T)(l < lmax ? Ac * kcur / knext : 0.0);
    tB[base + l] = (T)(l < lmax ? Bt * kcur / knext : 0.0);
    kprev = kcur;
    kcur = knext;
  }
}

// ---------------------------------------------------------------------------------------------
template <typename T>
struct Rc;
template <>
struct Rc<double> {
  __device__ __forceinline__ static bool big(double y) {
    return (__double2hiint(y) & 0x7fffffff) >= ((1023 + ScaleConst<double>::R_EXP) << 20);
  }
  __device__ __forceinline__ static double down() { return 0x1p-500; }
};
template <>
struct Rc<float> {
  __device__ __forceinline__ static bool big(float y) {
    return (__float_as_int(y) & 0x7fffffff) >= ((127 + ScaleConst<float>::R_EXP) << 23);
  }
  __device__ __forceinline__ static float down() { return 0x1p-80f; }
};
static_assert(ScaleConst<double>::F == 500, "down() hard-codes F");
static_assert(ScaleConst<float>::F == 80, "down() hard-codes F");

// seed y = sign 2^lg held as y 2^(-F k), from the FP64 log2 magnitude
template <typename T>
__device__ __forceinline__ void seed_scaled(double lg, int sign, T& y, int& k) {
  constexpr int F = ScaleConst<T>::F, RE = ScaleConst<T>::R_EXP;
  if (!(lg > -1.0e30)) {  // exact zero (a zero half-angle to a positive power)
    y = (T)0;
    k = 1;
    return;
  }
  if (lg >= (double)(RE - F)) {
    k = 0;
  } else {
    k = (int)ceil(((double)(RE - F) - lg) / (double)F);
    lg += (double)F * k;
  }
  y = (T)(sign * exp2(lg));
}

__device__ __forceinline__ double seed_log2(double lbin, int p, int q, double l2c, double l2s) {
  double v = lbin;
  if (p > 0) v += (double)p * l2c;
  if (q > 0) v += (double)q * l2s;
  return v;
}

template <typename T>
__device__ __forceinline__ T ring_ax(T A, const RingDev& r, T xr, T xlo);
template <>
__device__ __forceinline__ double ring_ax<double>(double A, const RingDev&, double x, double) {
  return A * x;
}
template <>
__device__ __forceinline__ float ring_ax<float>(float A, const RingDev&, float xhi, float xlo) {
  // x carried as xhi + xlo so that the ring position is exact to FP64 level
  return fmaf(A, xhi, A * xlo);
}

template <typename T>
__device__ __forceinline__ void ring_x(const RingDev& r, T& x, T& xlo);
template <>
__device__ __forceinline__ void ring_x<double>(const RingDev& r, double& x, double& xlo) {
  x = r.x;
  xlo = 0.0;
}
template <>
__device__ __forceinline__ void ring_x<float>(const RingDev& r, float& x, float& xlo) {
  x = r.xhi;
  xlo = r.xlo;
}

// ---------------------------------------------------------------------------------------------
// synthesis: one CTA per RecItem (order m, rings j0 .. j0+nj-1), RPT rings per thread.
template <typename T, bool SPIN, int RPT>
__global__ void __launch_bounds__(128) k_rec_syn(const RecItem* __restrict__ items, const RingDev* __restrict__ rings,
                                                 const MSeed* __restrict__ mseed, const T* __restrict__ tA,
                                                 const T* __restrict__ tB, const T* __restrict__ tK,
                                                 const typename Cx<T>::V* __restrict__ g,
                                                 const typename Cx<T>::V* __restrict__ c, int lmax, int s,
                                                 typename Cx<T>::V* __restrict__ F, int Lpad) {
  using V = typename Cx<T>::V;
  const RecItem it = items[blockIdx.x];
  const int m = it.m;
  const MSeed sd = mseed[m];
  __shared__ T sA[kCH], sB[kCH];
  __shared__ V sU[kCH], sV[kCH];

  T x[RPT], xlo[RPT], y1[RPT], y1p[RPT], y2[RPT], y2p[RPT];
  T a0[RPT], a1[RPT], a2[RPT], a3[RPT];
  int k1[RPT], k2[RPT];
  bool any = false;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = threadIdx.x + r * blockDim.x;
    a0[r] = a1[r] = a2[r] = a3[r] = (T)0;
    y1p[r] = y2p[r] = (T)0;
    if (jj < it.nj) {
      const RingDev rg = rings[it.j0 + jj];
      ring_x<T>(rg, x[r], xlo[r]);
      seed_scaled<T>(seed_log2(sd.lbin, sd.p1, sd.q1, rg.l2c, rg.l2s), sd.sign1, y1[r], k1[r]);
      if (SPIN) seed_scaled<T>(seed_log2(sd.lbin, sd.q1, sd.p1, rg.l2c, rg.l2s), sd.sign2, y2[r], k2[r]);
      any = true;
    } else {
      x[r] = xlo[r] = y1[r] = y2[r] = (T)0;
      k1[r] = k2[r] = 1;
    }
  }
  const bool warp_any = __any_sync(0xffffffffu, any);
  const int64_t base = alm_base(lmax, m);
  const bool m0 = (m == 0);

  for (int lc = sd.l0; lc <= lmax; lc += kCH) {
    const int n = min(kCH, lmax - lc + 1);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t id = base + lc + i;
      const T kap = tK[id];
      sA[i] = tA[id];
      sB[i] = tB[id];
      V gv = g[id];
      V cv = c ? c[id] : mk((T)0, (T)0);
      if (m0) {
        gv.y = (T)0;
        cv.y = (T)0;
      }
      sU[i] = mk(kap * (gv.x - cv.y), kap * (gv.y + cv.x));  // kappa (g + i c)
      sV[i] = mk(kap * (gv.x + cv.y), kap * (cv.x - gv.y));  // kappa (g* + i c*)
    }
    __syncthreads();
    if (!warp_any) continue;
    for (int i = 0; i < n; ++i) {
      const T A = sA[i], B = sB[i];
      const V u = sU[i], v = sV[i];
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const T o1 = (k1[r] == 0) ? y1[r] : (T)0;
        a0[r] = fma(u.x, o1, a0[r]);
        a1[r] = fma(u.y, o1, a1[r]);
        const T ax = ring_ax<T>(A, RingDev{}, x[r], xlo[r]);
        const T n1 = fma(ax + B, y1[r], -y1p[r]);
        y1p[r] = y1[r];
        y1[r] = n1;
        if (SPIN) {
          const T o2 = (k2[r] == 0) ? y2[r] : (T)0;
          a2[r] = fma(v.x, o2, a2[r]);
          a3[r] = fma(v.y, o2, a3[r]);
          const T n2 = fma(ax - B, y2[r], -y2p[r]);
          y2p[r] = y2[r];
          y2[r] = n2;
          if (k2[r] > 0 && Rc<T>::big(n2)) {
            y2[r] *= Rc<T>::down();
            y2p[r] *= Rc<T>::down();
            --k2[r];
          }
        } else {
          a2[r] = fma(v.x, o1, a2[r]);
          a3[r] = fma(v.y, o1, a3[r]);
        }
        if (k1[r] > 0 && Rc<T>::big(n1)) {
          y1[r] *= Rc<T>::down();
          y1p[r] *= Rc<T>::down();
          --k1[r];
        }
      }
    }
  }
  const T sgn_s = (s & 1) ? (T)1 : (T)-1;  // -(-1)^s
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = threadIdx.x + r * blockDim.x;
    if (jj < it.nj) {
      const int j = it.j0 + jj;
      F[(int64_t)col_of(m) * Lpad + j] = mk(-a0[r], -a1[r]);
      if (!m0) F[(int64_t)col_of(-m) * Lpad + j] = mk(sgn_s * a2[r], sgn_s * a3[r]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// adjoint: one CTA per order m (blockIdx.x = m), all active rings, RPT rings per thread.
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, bool SPIN, int RPT>
__global__ void __launch_bounds__(512) k_rec_adj(const RingDev* __restrict__ rings, const MSeed* __restrict__ mseed,
                                                 const int2* __restrict__ mrange, const T* __restrict__ tA,
                                                 const T* __restrict__ tB, const T* __restrict__ tK,
                                                 const typename Cx<T>::V* __restrict__ Ft, int Lpad, int lmax, int s,
                                                 int M, typename Cx<T>::V* __restrict__ gt,
                                                 typename Cx<T>::V* __restrict__ ct) {
  using V = typename Cx<T>::V;
  const int m = blockIdx.x;
  const int64_t base = alm_base(lmax, m);
  if (m > M) {  // beyond the polar-optimisation cutoff on every ring: exact transpose of a zero block
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      gt[base + l] = mk((T)0, (T)0);
      if (ct) ct[base + l] = mk((T)0, (T)0);
    }
    return;
  }
  const MSeed sd = mseed[m];
  const int2 rr = mrange[m];
  const int nact = rr.y - rr.x;
  constexpr int NW = 512 / 32;
  __shared__ T sA[kCH], sB[kCH], sK[kCH];
  __shared__ T red[NW][kCH][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  for (int l = m + threadIdx.x; l < sd.l0 && l <= lmax; l += blockDim.x) {
    gt[base + l] = mk((T)0, (T)0);
    if (ct) ct[base + l] = mk((T)0, (T)0);
  }

  T x[RPT], xlo[RPT], y1[RPT], y1p[RPT], y2[RPT], y2p[RPT];
  V fp[RPT], fm[RPT];
  int k1[RPT], k2[RPT];
  bool any = false;
  const bool m0 = (m == 0);
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = threadIdx.x + r * blockDim.x;
    y1p[r] = y2p[r] = (T)0;
    if (jj < nact) {
      const int j = rr.x + jj;
      const RingDev rg = rings[j];
      ring_x<T>(rg, x[r], xlo[r]);
      seed_scaled<T>(seed_log2(sd.lbin, sd.p1, sd.q1, rg.l2c, rg.l2s), sd.sign1, y1[r], k1[r]);
      if (SPIN) seed_scaled<T>(seed_log2(sd.lbin, sd.q1, sd.p1, rg.l2c, rg.l2s), sd.sign2, y2[r], k2[r]);
      fp[r] = Ft[(int64_t)col_of(m) * Lpad + j];
      fm[r] = m0 ? mk((T)0, (T)0) : Ft[(int64_t)col_of(-m) * Lpad + j];
      any = true;
    } else {
      x[r] = xlo[r] = y1[r] = y2[r] = (T)0;
      k1[r] = k2[r] = 1;
      fp[r] = fm[r] = mk((T)0, (T)0);
    }
  }
  const bool warp_any = __any_sync(0xffffffffu, any);
  const T sg = (((m - s) & 1) ? (T)1 : (T)-1);  // -(-1)^(m-s)
  const T sm = (m & 1) ? (T)-1 : (T)1;          // (-1)^m

  for (int lc = sd.l0; lc <= lmax; lc += kCH) {
    const int n = min(kCH, lmax - lc + 1);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t id = base + lc + i;
      sA[i] = tA[id];
      sB[i] = tB[id];
      sK[i] = tK[id];
    }
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      T p0 = 0, p1 = 0, p2 = 0, p3 = 0;
      if (warp_any) {
        const T A = sA[i], B = sB[i];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const T o1 = (k1[r] == 0) ? y1[r] : (T)0;
          p0 = fma(o1, fp[r].x, p0);
          p1 = fma(o1, fp[r].y, p1);
          const T ax = ring_ax<T>(A, RingDev{}, x[r], xlo[r]);
          const T n1 = fma(ax + B, y1[r], -y1p[r]);
          y1p[r] = y1[r];
          y1[r] = n1;
          if (SPIN) {
            const T o2 = (k2[r] == 0) ? y2[r] : (T)0;
            p2 = fma(o2, fm[r].x, p2);
            p3 = fma(o2, fm[r].y, p3);
            const T n2 = fma(ax - B, y2[r], -y2p[r]);
            y2p[r] = y2[r];
            y2[r] = n2;
            if (k2[r] > 0 && Rc<T>::big(n2)) {
              y2[r] *= Rc<T>::down();
              y2p[r] *= Rc<T>::down();
              --k2[r];
            }
          } else {
            p2 = fma(o1, fm[r].x, p2);
            p3 = fma(o1, fm[r].y, p3);
          }
          if (k1[r] > 0 && Rc<T>::big(n1)) {
            y1[r] *= Rc<T>::down();
            y1p[r] *= Rc<T>::down();
            --k1[r];
          }
        }
        p0 = warp_sum(p0);
        p1 = warp_sum(p1);
        p2 = warp_sum(p2);
        p3 = warp_sum(p3);
      }
      if (lane == 0) {
        red[warp][i][0] = p0;
        red[warp][i][1] = p1;
        red[warp][i][2] = p2;
        red[warp][i][3] = p3;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
      for (int w = 0; w < nwarps; ++w) {
        q0 += red[w][i][0];
        q1 += red[w][i][1];
        q2 += red[w][i][2];
        q3 += red[w][i][3];
      }
      const T kap = sK[i];
      // ut_{l,m} = -kappa (q0 + i q1);  ut_{l,-m} = -(-1)^(m-s) kappa (q2 + i q3)
      const T ar = -kap * q0, ai = -kap * q1;
      const T br = sg * kap * q2, bi = sg * kap * q3;
      const int64_t id = base + lc + i;
      if (m0) {
        gt[id] = mk(ar, (T)0);
        if (ct) ct[id] = mk(ai, (T)0);
      } else {
        const T wr = sm * br, wi = -sm * bi;  // (-1)^m conj(ut_{l,-m})
        gt[id] = mk((T)0.5 * (ar + wr), (T)0.5 * (ai + wi));
        if (ct) ct[id] = mk((T)0.5 * (ai - wi), (T)-0.5 * (ar - wr));
      }
    }
  }
}

template <typename T, bool SPIN, int RPT>
void launch_syn_t(Plan& p, const void* g, const void* c, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const T* tA = (const T*)p.d_rtab;
  const T* tB = tA + p.nalm;
  const T* tK = tB + p.nalm;
  k_rec_syn<T, SPIN, RPT><<<p.nitems, 128, 0, st>>>(p.d_items, p.d_ring, p.d_mseed, tA, tB, tK, (const V*)g,
                                                     (const V*)c, p.lmax, p.spin, (V*)p.d_F, p.Lpad);
}

template <typename T, bool SPIN, int RPT>
void launch_adj_t(Plan& p, void* g, void* c, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const T* tA = (const T*)p.d_rtab;
  const T* tB = tA + p.nalm;
  const T* tK = tB + p.nalm;
  k_rec_adj<T, SPIN, RPT><<<p.lmax + 1, p.adj_threads, 0, st>>>(p.d_ring, p.d_mseed, p.d_mrange, tA, tB, tK,
                                                                (const V*)p.d_F, p.Lpad, p.lmax, p.spin, p.M,
                                                                (V*)g, (V*)c);
}

template <typename T, bool SPIN>
void launch_syn_s(Plan& p, const void* g, const void* c, cudaStream_t st) {
  switch (p.syn_rpt) {
    case 1: launch_syn_t<T, SPIN, 1>(p, g, c, st); break;
    case 2: launch_syn_t<T, SPIN, 2>(p, g, c, st); break;
    default: launch_syn_t<T, SPIN, 4>(p, g, c, st); break;
  }
}
template <typename T, bool SPIN>
void launch_adj_s(Plan& p, void* g, void* c, cudaStream_t st) {
  switch (p.adj_rpt) {
    case 1: launch_adj_t<T, SPIN, 1>(p, g, c, st); break;
    case 2: launch_adj_t<T, SPIN, 2>(p, g, c, st); break;
    case 4: launch_adj_t<T, SPIN, 4>(p, g, c, st); break;
    default: launch_adj_t<T, SPIN, 8>(p, g, c, st); break;
  }
}

}  // namespace

void build_rec_table(Plan& p, cudaStream_t st) {
  const int nth = 128, nbl = (p.lmax + 1 + nth - 1) / nth;
  if (p.prec == 64) {
    double* t = (double*)p.d_rtab;
    k_rec_table<double><<<nbl, nth, 0, st>>>(p.lmax, p.spin, t, t + p.nalm, t + 2 * p.nalm);
  } else {
    float* t = (float*)p.d_rtab;
    k_rec_table<float><<<nbl, nth, 0, st>>>(p.lmax, p.spin, t, t + p.nalm, t + 2 * p.nalm);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_rec_synthesis(Plan& p, const void* g, const void* c, cudaStream_t st) {
  if (p.nitems == 0) return;
  if (p.prec == 64) {
    if (p.spin) launch_syn_s<double, true>(p, g, c, st);
    else launch_syn_s<double, false>(p, g, c, st);
  } else {
    if (p.spin) launch_syn_s<float, true>(p, g, c, st);
    else launch_syn_s<float, false>(p, g, c, st);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_rec_adjoint(Plan& p, void* g, void* c, cudaStream_t st) {
  if (p.prec == 64) {
    if (p.spin) launch_adj_s<double, true>(p, g, c, st);
    else launch_adj_s<double, false>(p, g, c, st);
  } else {
    if (p.spin) launch_adj_s<float, true>(p, g, c, st);
    else launch_adj_s<float, false>(p, g, c, st);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

}  // namespace psht
