// Wigner-d recursion onto the apodised rings (synthesis, "K-REC") and its transpose
// (adjoint, "K-REC-ADJ").
//
// Per order m and ring j the two columns e1_l = N_l d^l_{m,-s}(beta_j) and e2_l = N_l d^l_{m,s}(beta_j)
// (sY_lm = N_l d^l_{m,-s} e^{im phi}, appendix eq. Ylm; N_l = sqrt((2l+1)/4pi)) obey the textbook
// three-term recurrence in l, written for the normalised columns as
//     e_{l+1} = (A_l x +- B_l) e_l - C_l e_{l-1},   x = cos(beta_j),
// and evaluated in Reinsch's form for x near 1: with D_l = A_l - 1 - C_l and Delta_l = e_l - e_{l-1},
//     Delta_{l+1} = (D_l +- B_l - A_l (1 - x)) e_l + C_l Delta_l,   e_{l+1} = e_l + Delta_{l+1},
// where 1 - x = 2 sin^2(beta/2) is exact on the host.  This keeps the recurrence accurate on the
// rings next to the pole, where A x + B - 2 is far below the rounding of A x + B.  In the FP32
// form A, D and 1 - x are carried as float pairs (hi + lo).
// Rings of a south-pole plan sit at theta_j = pi - beta_j; they are evaluated at beta_j with
// d^l_{m,-s}(pi - beta) = (-1)^(l+m) d^l_{m,s}(beta), i.e. with the two columns swapped and the
// coefficients signed by (-1)^(l+m).
// Seeds are Wigner's closed form at l0 = max(m, s) in FP64 log2 form; values too small for the
// working precision are carried as e 2^(-F k) and join the sums once k = 0.
//
// Synthesis (eq. syn on ring j):   F_j[m] = -sum_l (g + i c)_lm e1_l,   F_j[-m] = -(-1)^s sum_l (g* + i c*)_lm e2_l
// Adjoint (transpose, then the projection of the adjoint synthesis general formula, Sec. I):
//   ut_{l,m} = -sum_j e1_l(j) Ft_j[m],   ut_{l,-m} = -(-1)^(m-s) sum_j e2_l(j) Ft_j[-m]
//   g~ = (ut_lm + (-1)^m conj ut_{l,-m})/2,   c~ = (ut_lm - (-1)^m conj ut_{l,-m})/(2i)
#include <cuda_runtime.h>
#include <math.h>

#include "psht_common.cuh"

namespace psht {

namespace {

constexpr int kCH = 64;  // l values staged in shared memory per chunk

__device__ __forceinline__ int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// ---------------------------------------------------------------------------------------------
// recurrence table per packed (l, m), FP64 arithmetic, one thread per m.
//   FP64 form: t[0] = A, t[1] = D, t[2] = B, t[3] = C
//   FP32 form: t[0] = A_hi, t[1] = A_lo, t[2] = D_hi, t[3] = D_lo, t[4] = B, t[5] = C
template <typename T>
__global__ void k_rec_table(int lmax, int s, T* __restrict__ tab, int64_t nalm) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > lmax) return;
  const int l0 = max(m, s);
  const int64_t base = alm_base(lmax, m);
  const double m2 = (double)m * m, s2 = (double)s * s;
  for (int l = m; l <= lmax; ++l) {
    double A = 0, B = 0, C = 0, D = 0;
    if (l >= l0 && l < lmax) {
      const double lp1 = l + 1.0;
      const double a = lp1 * (2.0 * l + 1.0) / sqrt((lp1 * lp1 - m2) * (lp1 * lp1 - s2));
      A = sqrt((2.0 * l + 3.0) / (2.0 * l + 1.0)) * a;
      B = (l == 0) ? 0.0 : A * (double)m * (double)s / ((double)l * lp1);
      if (l > l0) {
        const double c = sqrt(((double)l * l - m2) * ((double)l * l - s2)) / ((double)l * (2.0 * l + 1.0));
        C = sqrt((2.0 * l + 3.0) / (2.0 * l - 1.0)) * a * c;
      }
      D = (A - 1.0) - C;
    }
    const int64_t id = base + l;
    if (sizeof(T) == 8) {
      tab[id] = (T)A;
      tab[nalm + id] = (T)D;
      tab[2 * nalm + id] = (T)B;
      tab[3 * nalm + id] = (T)C;
    } else {
      const float ah = (float)A, dh = (float)D;
      tab[id] = ah;
      tab[nalm + id] = (float)(A - (double)ah);
      tab[2 * nalm + id] = dh;
      tab[3 * nalm + id] = (float)(D - (double)dh);
      tab[4 * nalm + id] = (float)B;
      tab[5 * nalm + id] = (float)C;
    }
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

// staged recurrence coefficients of one l, and the shared part t = D - A (1 - x) of the multiplier
template <typename T>
struct Coef;
template <>
struct Coef<double> {
  double A, D, B, C;
  __device__ __forceinline__ double t(double omx, double) const { return fma(-A, omx, D); }
};
template <>
struct Coef<float> {
  float Ah, Al, Dh, Dl, B, C;
  __device__ __forceinline__ float t(float oh, float ol) const {
    return fmaf(-Ah, oh, Dh) + fmaf(-Ah, ol, fmaf(-Al, oh, Dl));
  }
};

template <typename T>
__device__ __forceinline__ Coef<T> load_coef(const T* __restrict__ tab, int64_t nalm, int64_t id);
template <>
__device__ __forceinline__ Coef<double> load_coef<double>(const double* __restrict__ tab, int64_t nalm, int64_t id) {
  return Coef<double>{tab[id], tab[nalm + id], tab[2 * nalm + id], tab[3 * nalm + id]};
}
template <>
__device__ __forceinline__ Coef<float> load_coef<float>(const float* __restrict__ tab, int64_t nalm, int64_t id) {
  return Coef<float>{tab[id], tab[nalm + id], tab[2 * nalm + id], tab[3 * nalm + id], tab[4 * nalm + id],
                     tab[5 * nalm + id]};
}

template <typename T>
__device__ __forceinline__ void ring_omx(const RingDev& r, T& oh, T& ol);
template <>
__device__ __forceinline__ void ring_omx<double>(const RingDev& r, double& oh, double& ol) {
  oh = r.omx;
  ol = 0.0;
}
template <>
__device__ __forceinline__ void ring_omx<float>(const RingDev& r, float& oh, float& ol) {
  oh = r.ohi;
  ol = r.olo;
}

// one Reinsch step of a column: Delta <- t e + C Delta, e <- e + Delta
template <typename T>
__device__ __forceinline__ void reinsch_step(T t, T C, T& e, T& d) {
  d = fma(t, e, C * d);
  e = e + d;
}
// rescale guard, run once per quad of l steps while a column is in its dropped region
template <typename T>
__device__ __forceinline__ void rescale(T& e, T& d, int& k) {
  if (k > 0 && Rc<T>::big(e)) {
    e *= Rc<T>::down();
    d *= Rc<T>::down();
    --k;
  }
}

// staged a_lm combination for the two columns: direct rings P = g + i c (col 1), Q = g* + i c* (col 2);
// reflected rings P = (-1)^(l+m) (g* + i c*), Q = (-1)^(l+m) (g + i c)
template <typename V, typename T>
__device__ __forceinline__ void stage_pq(V gv, V cv, bool m0, bool refl, int lpm, V& P, V& Q) {
  if (m0) {
    gv.y = (T)0;
    cv.y = (T)0;
  }
  V u = mk(gv.x - cv.y, gv.y + cv.x);
  V v = mk(gv.x + cv.y, cv.x - gv.y);
  if (refl) {
    const T sg = (lpm & 1) ? (T)-1 : (T)1;
    P = mk(sg * v.x, sg * v.y);
    Q = mk(sg * u.x, sg * u.y);
  } else {
    P = u;
    Q = v;
  }
}

// Shared-memory staging of one chunk of l values.  Entries past lmax get zero coefficients, which
// leave the state unchanged and add nothing, so every chunk is a whole number of quads.
template <typename T>
struct Stage {
  Coef<T> cf[kCH];
  typename Cx<T>::V P[kCH], Q[kCH];
};

template <typename T, bool WITH_PQ>
__device__ __forceinline__ void stage_chunk(Stage<T>& S, const T* __restrict__ tab, int64_t nalm, int64_t base,
                                            int lc, int lmax, int m,
                                            const typename Cx<T>::V* __restrict__ g,
                                            const typename Cx<T>::V* __restrict__ c, bool refl) {
  using V = typename Cx<T>::V;
  for (int i = threadIdx.x; i < kCH; i += blockDim.x) {
    const int l = lc + i;
    if (l <= lmax) {
      const int64_t id = base + l;
      S.cf[i] = load_coef<T>(tab, nalm, id);
      if (WITH_PQ) {
        V P, Q;
        stage_pq<V, T>(g[id], c ? c[id] : mk((T)0, (T)0), m == 0, refl, l + m, P, Q);
        S.P[i] = P;
        S.Q[i] = Q;
      }
    } else {
      S.cf[i] = Coef<T>{};
      if (WITH_PQ) {
        S.P[i] = mk((T)0, (T)0);
        S.Q[i] = mk((T)0, (T)0);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// synthesis: one CTA per RecItem (order m, rings j0 .. j0+nj-1), RPT rings per thread.
// Work proceeds in quads of 4 l steps; per quad each warp takes one of three uniform paths:
// all its columns past the dropped region (no tests), all still inside it (no sums), or mixed.
template <typename T, bool SPIN, int RPT>
__global__ void __launch_bounds__(128) k_rec_syn(const RecItem* __restrict__ items, const RingDev* __restrict__ rings,
                                                 const MSeed* __restrict__ mseed, const T* __restrict__ tab,
                                                 int64_t nalm, const typename Cx<T>::V* __restrict__ g,
                                                 const typename Cx<T>::V* __restrict__ c, int lmax, int s,
                                                 typename Cx<T>::V* __restrict__ F, int Lpad) {
  using V = typename Cx<T>::V;
  const RecItem it = items[blockIdx.x];
  const int m = it.m;
  const MSeed sd = mseed[m];
  __shared__ Stage<T> S;

  T oh[RPT], ol[RPT], e1[RPT], d1[RPT], e2[RPT], d2[RPT];
  T a0[RPT], a1[RPT], a2[RPT], a3[RPT];
  int k1[RPT], k2[RPT];
  bool any = false;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = threadIdx.x + r * blockDim.x;
    a0[r] = a1[r] = a2[r] = a3[r] = (T)0;
    if (jj < it.nj) {
      const RingDev rg = rings[it.j0 + jj];
      ring_omx<T>(rg, oh[r], ol[r]);
      seed_scaled<T>(seed_log2(sd.lbin, sd.p1, sd.q1, rg.l2c, rg.l2s), sd.sign1, e1[r], k1[r]);
      if (SPIN) seed_scaled<T>(seed_log2(sd.lbin, sd.q1, sd.p1, rg.l2c, rg.l2s), sd.sign2, e2[r], k2[r]);
      else k2[r] = 0;
      any = true;
    } else {
      oh[r] = ol[r] = e1[r] = e2[r] = (T)0;
      k1[r] = 1;
      k2[r] = SPIN ? 1 : 0;
    }
    d1[r] = e1[r];  // Delta_{l0} = e_{l0} - e_{l0-1}, e_{l0-1} = 0
    d2[r] = e2[r];
  }
  const bool warp_any = __any_sync(0xffffffffu, any);
  const int64_t base = alm_base(lmax, m);
  const bool rf = it.refl != 0;

  for (int lc = sd.l0; lc <= lmax; lc += kCH) {
    __syncthreads();
    stage_chunk<T, true>(S, tab, nalm, base, lc, lmax, m, g, c, rf);
    __syncthreads();
    if (!warp_any) continue;
    const int nq = (min(kCH, lmax - lc + 1) + 3) >> 2;
    for (int q = 0; q < nq; ++q) {
      bool in2 = true, in1 = true;  // all columns summing / all columns still dropped
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        in2 = in2 && k1[r] == 0 && k2[r] == 0;
        in1 = in1 && k1[r] > 0 && (!SPIN || k2[r] > 0);
      }
      const bool fast = __all_sync(0xffffffffu, in2);
      const bool skip = !fast && __all_sync(0xffffffffu, in1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 4 * q + u;
        const Coef<T> cf = S.cf[i];
        const V P = S.P[i], Q = S.Q[i];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if (!skip) {
            const T o1 = (fast || k1[r] == 0) ? e1[r] : (T)0;
            a0[r] = fma(P.x, o1, a0[r]);
            a1[r] = fma(P.y, o1, a1[r]);
            if (SPIN) {
              const T o2 = (fast || k2[r] == 0) ? e2[r] : (T)0;
              a2[r] = fma(Q.x, o2, a2[r]);
              a3[r] = fma(Q.y, o2, a3[r]);
            } else {
              a2[r] = fma(Q.x, o1, a2[r]);
              a3[r] = fma(Q.y, o1, a3[r]);
            }
          }
          const T t = cf.t(oh[r], ol[r]);
          if (SPIN) {
            reinsch_step<T>(t + cf.B, cf.C, e1[r], d1[r]);
            reinsch_step<T>(t - cf.B, cf.C, e2[r], d2[r]);
          } else {
            reinsch_step<T>(t, cf.C, e1[r], d1[r]);
          }
        }
      }
      if (!fast) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          rescale<T>(e1[r], d1[r], k1[r]);
          if (SPIN) rescale<T>(e2[r], d2[r], k2[r]);
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
      // direct rings: F[m] <- column 1, F[-m] <- column 2; reflected rings: swapped
      const V fpos = rf ? mk(-a2[r], -a3[r]) : mk(-a0[r], -a1[r]);
      const V fneg = rf ? mk(sgn_s * a0[r], sgn_s * a1[r]) : mk(sgn_s * a2[r], sgn_s * a3[r]);
      F[(int64_t)col_of(m) * Lpad + j] = fpos;
      if (m != 0) F[(int64_t)col_of(-m) * Lpad + j] = fneg;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// adjoint: one CTA per order m (blockIdx.x = m), the active rings of one ring part, RPT rings
// per thread.  Per quad the 4 l values x 4 partial sums of each thread are reduced across the
// warp by a reduce-scatter (16 values over 32 lanes: 4 halving exchanges and one final add).
template <typename T>
__device__ __forceinline__ T reduce_scatter16(T (&v)[16], int lane) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const T send = up ? v[k] : v[k + o];
      const T keep = up ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);  // lane holds value (lane & 15)
}

template <typename T, bool SPIN, int RPT, int NT>
__global__ void __launch_bounds__(NT) k_rec_adj(const RingDev* __restrict__ rings, const MSeed* __restrict__ mseed,
                                                const int2* __restrict__ mrange, const T* __restrict__ tab,
                                                int64_t nalm, const typename Cx<T>::V* __restrict__ Ft, int Lpad,
                                                int lmax, int s, int M, int refl, int accumulate,
                                                typename Cx<T>::V* __restrict__ gt,
                                                typename Cx<T>::V* __restrict__ ct) {
  using V = typename Cx<T>::V;
  const int m = blockIdx.x;
  const int64_t base = alm_base(lmax, m);
  if (m > M) {  // beyond the polar-optimisation cutoff on every ring: transpose of a zero block
    if (accumulate) return;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      gt[base + l] = mk((T)0, (T)0);
      if (ct) ct[base + l] = mk((T)0, (T)0);
    }
    return;
  }
  const MSeed sd = mseed[m];
  const int2 rr = mrange[m];
  const int nact = rr.y - rr.x;
  constexpr int NW = NT / 32;
  __shared__ Stage<T> S;
  __shared__ T red[NW][kCH][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int l = m + threadIdx.x; !accumulate && l < sd.l0 && l <= lmax; l += blockDim.x) {
    gt[base + l] = mk((T)0, (T)0);
    if (ct) ct[base + l] = mk((T)0, (T)0);
  }
  const bool m0 = (m == 0);
  const bool rf = refl != 0;

  T oh[RPT], ol[RPT], e1[RPT], d1[RPT], e2[RPT], d2[RPT];
  V f1[RPT], f2[RPT];  // ring values paired with column 1 / column 2
  int k1[RPT], k2[RPT];
  bool any = false;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = threadIdx.x + r * blockDim.x;
    if (jj < nact) {
      const int j = rr.x + jj;
      const RingDev rg = rings[j];
      ring_omx<T>(rg, oh[r], ol[r]);
      seed_scaled<T>(seed_log2(sd.lbin, sd.p1, sd.q1, rg.l2c, rg.l2s), sd.sign1, e1[r], k1[r]);
      if (SPIN) seed_scaled<T>(seed_log2(sd.lbin, sd.q1, sd.p1, rg.l2c, rg.l2s), sd.sign2, e2[r], k2[r]);
      else k2[r] = 0;
      const V fp = Ft[(int64_t)col_of(m) * Lpad + j];
      const V fm = m0 ? mk((T)0, (T)0) : Ft[(int64_t)col_of(-m) * Lpad + j];
      f1[r] = rf ? fm : fp;
      f2[r] = rf ? fp : fm;
      any = true;
    } else {
      oh[r] = ol[r] = e1[r] = e2[r] = (T)0;
      k1[r] = 1;
      k2[r] = SPIN ? 1 : 0;
      f1[r] = f2[r] = mk((T)0, (T)0);
    }
    d1[r] = e1[r];
    d2[r] = e2[r];
  }
  const bool warp_any = __any_sync(0xffffffffu, any);
  const T sg = (((m - s) & 1) ? (T)1 : (T)-1);  // -(-1)^(m-s)
  const T sm = (m & 1) ? (T)-1 : (T)1;          // (-1)^m

  for (int lc = sd.l0; lc <= lmax; lc += kCH) {
    const int n = min(kCH, lmax - lc + 1);
    const int nq = (n + 3) >> 2;
    __syncthreads();
    stage_chunk<T, false>(S, tab, nalm, base, lc, lmax, m, nullptr, nullptr, rf);
    __syncthreads();
    for (int q = 0; q < nq; ++q) {
      if (!warp_any) {
        if (lane < 16) red[warp][4 * q + (lane >> 2)][lane & 3] = (T)0;
        continue;
      }
      bool in2 = true, in1 = true;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        in2 = in2 && k1[r] == 0 && k2[r] == 0;
        in1 = in1 && k1[r] > 0 && (!SPIN || k2[r] > 0);
      }
      const bool fast = __all_sync(0xffffffffu, in2);
      const bool skip = !fast && __all_sync(0xffffffffu, in1);
      T v[16];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const Coef<T> cf = S.cf[4 * q + u];
        T p0 = 0, p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if (!skip) {
            const T o1 = (fast || k1[r] == 0) ? e1[r] : (T)0;
            p0 = fma(o1, f1[r].x, p0);
            p1 = fma(o1, f1[r].y, p1);
            const T o2 = SPIN ? ((fast || k2[r] == 0) ? e2[r] : (T)0) : o1;
            p2 = fma(o2, f2[r].x, p2);
            p3 = fma(o2, f2[r].y, p3);
          }
          const T t = cf.t(oh[r], ol[r]);
          if (SPIN) {
            reinsch_step<T>(t + cf.B, cf.C, e1[r], d1[r]);
            reinsch_step<T>(t - cf.B, cf.C, e2[r], d2[r]);
          } else {
            reinsch_step<T>(t, cf.C, e1[r], d1[r]);
          }
        }
        v[4 * u + 0] = p0;
        v[4 * u + 1] = p1;
        v[4 * u + 2] = p2;
        v[4 * u + 3] = p3;
      }
      if (!fast) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          rescale<T>(e1[r], d1[r], k1[r]);
          if (SPIN) rescale<T>(e2[r], d2[r], k2[r]);
        }
      }
      if (skip) {
        if (lane < 16) red[warp][4 * q + (lane >> 2)][lane & 3] = (T)0;
      } else {
        const T tot = reduce_scatter16<T>(v, lane);
        if (lane < 16) red[warp][4 * q + (lane >> 2)][lane & 3] = tot;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        q0 += red[w][i][0];
        q1 += red[w][i][1];
        q2 += red[w][i][2];
        q3 += red[w][i][3];
      }
      const int l = lc + i;
      // sums against d_{m,-s}(theta) (Qp) and d_{m,s}(theta) (Qm); reflected rings swap the columns
      // and carry (-1)^(l+m)
      T Qpr = q0, Qpi = q1, Qmr = q2, Qmi = q3;
      if (rf) {
        const T sl = ((l + m) & 1) ? (T)-1 : (T)1;
        Qpr = sl * q2;
        Qpi = sl * q3;
        Qmr = sl * q0;
        Qmi = sl * q1;
      }
      // ut_{l,m} = -Qp;  ut_{l,-m} = -(-1)^(m-s) Qm
      const T ar = -Qpr, ai = -Qpi;
      const T br = sg * Qmr, bi = sg * Qmi;
      const int64_t id = base + l;
      V gv, cv;
      if (m0) {
        gv = mk(ar, (T)0);
        cv = mk(ai, (T)0);
      } else {
        const T wr = sm * br, wi = -sm * bi;  // (-1)^m conj(ut_{l,-m})
        gv = mk((T)0.5 * (ar + wr), (T)0.5 * (ai + wi));
        cv = mk((T)0.5 * (ai - wi), (T)-0.5 * (ar - wr));
      }
      if (accumulate) {  // the projection is linear: the second ring part adds its share
        gv = cadd(gv, gt[id]);
        if (ct) cv = cadd(cv, ct[id]);
      }
      gt[id] = gv;
      if (ct) ct[id] = cv;
    }
  }
}

template <typename T, bool SPIN, int RPT>
void launch_syn_t(Plan& p, const void* g, const void* c, cudaStream_t st) {
  using V = typename Cx<T>::V;
  k_rec_syn<T, SPIN, RPT><<<p.nitems, 128, 0, st>>>(p.d_items, p.d_ring, p.d_mseed, (const T*)p.d_rtab, p.nalm,
                                                     (const V*)g, (const V*)c, p.lmax, p.spin, (V*)p.d_F, p.Lpad);
}

template <typename T, bool SPIN, int RPT, int NT>
void launch_adj_t(Plan& p, void* g, void* c, cudaStream_t st) {
  using V = typename Cx<T>::V;
  // one launch per ring part (rings at theta <= pi/2, then reflected rings at theta > pi/2)
  for (int part = 0; part < 2; ++part) {
    if (part == 1 && !p.has_refl) break;
    k_rec_adj<T, SPIN, RPT, NT><<<p.lmax + 1, NT, 0, st>>>(
        p.d_ring, p.d_mseed, p.d_mrange + part * (p.lmax + 1), (const T*)p.d_rtab, p.nalm, (const V*)p.d_F, p.Lpad,
        p.lmax, p.spin, p.M, part, part, (V*)g, (V*)c);
  }
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
  // (rings per thread, threads) covering up to 4096 rings; chosen by the planner
  switch (p.adj_rpt * 10000 + p.adj_threads) {
    case 10128: launch_adj_t<T, SPIN, 1, 128>(p, g, c, st); break;
    case 20128: launch_adj_t<T, SPIN, 2, 128>(p, g, c, st); break;
    case 40128: launch_adj_t<T, SPIN, 4, 128>(p, g, c, st); break;
    case 40256: launch_adj_t<T, SPIN, 4, 256>(p, g, c, st); break;
    case 80128: launch_adj_t<T, SPIN, 8, 128>(p, g, c, st); break;
    case 80256: launch_adj_t<T, SPIN, 8, 256>(p, g, c, st); break;
    default: launch_adj_t<T, SPIN, 8, 512>(p, g, c, st); break;
  }
}

}  // namespace

int rec_table_width(int prec) { return prec == 64 ? 4 : 6; }

void build_rec_table(Plan& p, cudaStream_t st) {
  const int nth = 128, nbl = (p.lmax + 1 + nth - 1) / nth;
  if (p.prec == 64) k_rec_table<double><<<nbl, nth, 0, st>>>(p.lmax, p.spin, (double*)p.d_rtab, p.nalm);
  else k_rec_table<float><<<nbl, nth, 0, st>>>(p.lmax, p.spin, (float*)p.d_rtab, p.nalm);
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
