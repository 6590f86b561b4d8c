// Wigner-d recursion onto the apodised rings (synthesis, "K-REC") and its transpose
// (adjoint, "K-REC-ADJ").
//
// Per order m and ring j the two columns e1_l = N_l d^l_{m,-s}(b_j) and e2_l = N_l d^l_{m,s}(b_j)
// (sY_lm = N_l d^l_{m,-s} e^{im phi}, appendix eq. Ylm; N_l = sqrt((2l+1)/4pi)) obey the textbook
// three-term recurrence in l, written for the normalised columns as
//     e_{l+1} = (A_l x +- B_l) e_l - C_l e_{l-1},   x = cos(b_j),
// and evaluated in Reinsch's form for x near 1: with D_l = A_l - 1 - C_l and Delta_l = e_l - e_{l-1},
//     Delta_{l+1} = (D_l +- B_l - A_l (1 - x)) e_l + C_l Delta_l,   e_{l+1} = e_l + Delta_{l+1},
// where 1 - x = 2 sin^2(b/2) is exact on the host.  This keeps the recurrence accurate on the
// rings next to the pole, where A x + B - 2 is far below the rounding of A x + B.  In the FP32
// form A, D and 1 - x are carried as float pairs (hi + lo).  In the FP64 form, warps whose rings
// all lie at least kThreeTermDeg from the pole take the three-term form itself (two FP64
// operations per column and step instead of three; a few 1e-13 from Reinsch's there), when
// eps >= kThreeTermMinEps.
// Every ring is evaluated at b = min(theta_j, pi - theta_j): a ring at theta_j > pi/2 uses
// d^l_{m,-s}(pi - b) = (-1)^(l+m) d^l_{m,s}(b), i.e. the two columns swapped and the
// coefficients signed by (-1)^(l+m).
// Seeds are Wigner's closed form at l0 = max(m, s) in FP64 log2 form; values too small for the
// working precision are carried as e 2^(-F k) and join the sums once k = 0.  The one-warp kernels
// start each item at the first quad of l in which any of its columns has joined: the plan steps
// the quads below it once (k_rec_start) and keeps the columns' state there.
//
// Synthesis (eq. syn on ring j):   F_j[m] = -sum_l (g + i c)_lm e1_l,   F_j[-m] = -(-1)^s sum_l (g* + i c*)_lm e2_l
// Adjoint (transpose, then the projection of the adjoint synthesis general formula, Sec. I):
//   ut_{l,m} = -sum_j e1_l(j) Ft_j[m],   ut_{l,-m} = -(-1)^(m-s) sum_j e2_l(j) Ft_j[-m]
//   g~ = (ut_lm + (-1)^m conj ut_{l,-m})/2,   c~ = (ut_lm - (-1)^m conj ut_{l,-m})/(2i)
//
// Data movement: the recurrence table of an item's order m is streamed through shared memory by
// TMA bulk copies (cp.async.bulk, completion on an mbarrier, every wait bounded).  The one-warp
// kernels (k_rec_syn_w, k_rec_adj_w) copy chunks of 32 l with four stages in flight and prefetch
// the a_lm one chunk ahead through registers; the FP64 block adjoint (k_rec_adj) copies chunks of
// 64 l with two stages in flight.
//
// Kernels: k_rec_syn_w (synthesis, both forms; NS a_lm sets per pass, or mirror pairs of full-sky
// plans), k_rec_adj_w (FP32 adjoint; NS sets, or mirror pairs), k_rec_adj (FP64 adjoint, one CTA per
// order; mirror-pair orders in launches of their own), k_rec_table (the recurrence table),
// k_rec_start (the items' start states, plan time).
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "psht_common.cuh"

namespace psht {

namespace {

constexpr int kCH = 64;              // l values per chunk

__device__ __forceinline__ int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

struct alignas(32) Dbl4 {
  double x, y, z, w;
};
template <typename T>
struct Cx4;
template <>
struct Cx4<double> {
  using V = Dbl4;
};
template <>
struct Cx4<float> {
  using V = float4;
};

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// One record of the recurrence table per packed (l, m), so that a chunk of l values is one
// contiguous bulk copy and one l is a few vector shared-memory loads.  The FP32 form works on pairs of rings
// with packed FP32x2 instructions, so its record holds every coefficient twice (one per ring of
// the pair) and A negated: the packed operands come straight from shared memory.
template <typename T>
struct TabEntry;
template <>
struct TabEntry<float> {
  float4 na;  // -A_hi, -A_hi, -A_lo, -A_lo
  float4 d;   // D_hi, D_hi, D_lo, D_lo
  float4 bc;  // B, B, C, C
};
template <>
struct TabEntry<double> {
  double2 ad;  // A, D + B  (the Reinsch multiplier of column 1 is D + B - A (1 - x))
  double2 bc;  // D - B, C  (column 2: D - B - A (1 - x))
  double2 bz;  // B, 0      (three-term form: multipliers A x +- B)
};
static_assert(sizeof(TabEntry<float>) == 48 && sizeof(TabEntry<double>) == 48, "table record sizes");
static_assert((kCH * sizeof(TabEntry<float>)) % 16 == 0 && (kCH * sizeof(TabEntry<double>)) % 16 == 0,
              "bulk copies are whole 16-byte units");

// ---------------------------------------------------------------------------------------------
// recurrence table per packed (l, m), FP64 arithmetic: every record is a closed form in (l, m, s),
// so one thread per record; blockIdx.x = m, threads over l = m + blockIdx.y * blockDim.x + t.
template <typename T>
__global__ void k_rec_table(int lmax, int s, TabEntry<T>* __restrict__ tab) {
  const int m = blockIdx.x;
  const int l = m + blockIdx.y * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int l0 = max(m, s);
  const int64_t base = alm_base(lmax, m);
  const double m2 = (double)m * m, s2 = (double)s * s;
  {
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
    TabEntry<T> e;
    if constexpr (sizeof(T) == 8) {
      e.ad = make_double2(A, D + B);
      e.bc = make_double2(D - B, C);
      e.bz = make_double2(B, 0.0);
    } else {
      const float ah = (float)A, dh = (float)D;
      const float al = (float)(A - (double)ah), dl = (float)(D - (double)dh), b = (float)B, c = (float)C;
      e.na = make_float4(-ah, -ah, -al, -al);
      e.d = make_float4(dh, dh, dl, dl);
      e.bc = make_float4(b, b, c, c);
    }
    tab[base + l] = e;
  }
}

// ---------------------------------------------------------------------------------------------
// One staged chunk of the table: records of l = lc .. lc + 63 (zero records past lmax).
template <typename T, int CH = kCH>
struct TabStage {
  TabEntry<T> v[CH];
};

// Issue the bulk copy of table records start .. start + 63 into st (one thread).  The table is
// padded by one chunk of zero records, so the last chunk never reads past the allocation.
template <typename T, int CH = kCH>
__device__ __forceinline__ void issue_chunk(TabStage<T, CH>& st, uint64_t* bar, const TabEntry<T>* __restrict__ tab,
                                            int64_t start) {
  constexpr uint32_t bytes = CH * sizeof(TabEntry<T>);
  fence_proxy_async();  // earlier generic reads of this stage before the async-proxy writes
  mbar_expect_tx(bar, bytes);
  bulk_g2s(st.v, tab + start, bytes, bar);
}

// FP64 coefficients of one l; the column multipliers are D +- B - A (1 - x)
struct Coef {
  double A, DP, DM, C, B;  // A, D + B, D - B, C, B
  // Reinsch multipliers of the two columns (s = 0: B = 0 and only tp is used); one FMA each
  __device__ __forceinline__ double tp(double omx) const { return fma(-A, omx, DP); }
  __device__ __forceinline__ double tm(double omx) const { return fma(-A, omx, DM); }
  // three-term multipliers A x + B, A x - B
  __device__ __forceinline__ double up(double x) const { return fma(A, x, B); }
  __device__ __forceinline__ double um(double x) const { return fma(A, x, -B); }
};
__device__ __forceinline__ Coef get_coef(const TabEntry<double>* tv, int i) {
  const double2 ad = tv[i].ad, bc = tv[i].bc, bz = tv[i].bz;
  return Coef{ad.x, ad.y, bc.x, bc.y, bz.x};
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
__device__ __forceinline__ void reinsch_step(double t, double C, double& e, double& d) {
  d = fma(t, e, C * d);
  e = e + d;
}
// one step of the three-term form, e_{l+1} = u e_l - C e_{l-1}, with ep holding e_{l-1}: two FP64
// operations instead of Reinsch's three, exact to a few 1e-13 away from the pole but not next to it
// (u = A x +- B loses 1 - x there); used in FP64 on rings at least kThreeTermDeg from the pole
__device__ __forceinline__ void three_term_step(double u, double C, double& e, double& ep) {
  const double n = fma(u, e, -(C * ep));
  ep = e;
  e = n;
}
// both columns of one ring slot, one l step (oh: 1 - x for Reinsch, x for the three-term form)
template <bool SPIN, bool TB>
__device__ __forceinline__ void col_steps(const Coef& cf, double oh, double& e1, double& d1, double& e2, double& d2) {
  if (TB) {
    three_term_step(cf.up(oh), cf.C, e1, d1);
    if (SPIN) three_term_step(cf.um(oh), cf.C, e2, d2);
  } else {
    reinsch_step(cf.tp(oh), cf.C, e1, d1);
    if (SPIN) reinsch_step(cf.tm(oh), cf.C, e2, d2);
  }
}
// the same step for the two rings of a pair in packed FP32x2 arithmetic (per element the same
// roundings as the scalar step)
__device__ __forceinline__ void reinsch_step2(float2 t, float2 C, float2& e, float2& d) {
  d = __ffma2_rn(t, e, __fmul2_rn(C, d));
  e = __fadd2_rn(e, d);
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

// a_lm combination for the two columns: direct rings P = g + i c (col 1), Q = g* + i c* (col 2);
// reflected rings P = (-1)^(l+m) (g* + i c*), Q = (-1)^(l+m) (g + i c).  msc weights the m > 0
// entries (1, or 1/2 for the packed-gradient form; both exact).
template <typename V, typename T>
__device__ __forceinline__ void make_pq(V gv, V cv, bool m0, bool refl, int lpm, T msc, V& P, V& Q) {
  if (m0) {
    gv.y = (T)0;
    cv.y = (T)0;
  }
  const T w = m0 ? (T)1 : msc;
  V u = mk(w * (gv.x - cv.y), w * (gv.y + cv.x));
  V v = mk(w * (gv.x + cv.y), w * (cv.x - gv.y));
  if (refl) {
    const T sg = (lpm & 1) ? (T)-1 : (T)1;
    P = mk(sg * v.x, sg * v.y);
    Q = mk(sg * u.x, sg * u.y);
  } else {
    P = u;
    Q = v;
  }
}

// Shared-memory record of P and Q for one l.  FP64: (P.x, P.y, Q.x, Q.y).  FP32: every value
// twice, once per ring of a packed pair: (P.x, P.x, P.y, P.y), (Q.x, Q.x, Q.y, Q.y).
struct PQ2 {
  float4 p, q;
};
template <typename T>
struct PQRec;
template <>
struct PQRec<double> {
  using V = Dbl4;
};
template <>
struct PQRec<float> {
  using V = PQ2;
};
__device__ __forceinline__ Dbl4 pq_rec(double2 P, double2 Q) { return Dbl4{P.x, P.y, Q.x, Q.y}; }
__device__ __forceinline__ PQ2 pq_rec(float2 P, float2 Q) {
  return PQ2{make_float4(P.x, P.x, P.y, P.y), make_float4(Q.x, Q.x, Q.y, Q.y)};
}

// Per-thread state of RPT ring slots: 1 - x (hi + lo), the two columns e, their differences
// Delta, and the scale counts.  FP64 keeps one value per slot.  FP32 keeps slots 2p and 2p + 1 in
// one float2, the operand shape of the packed FP32x2 instructions, so that every arithmetic
// instruction of a step serves two rings.  The accessors give the value of one slot.
template <typename T, int RPT>
struct Cols {
  T oh[RPT], ol[RPT], e1[RPT], d1[RPT], e2[RPT], d2[RPT];
  int k1[RPT], k2[RPT];
  __device__ __forceinline__ T& OH(int r) { return oh[r]; }
  __device__ __forceinline__ T& OL(int r) { return ol[r]; }
  __device__ __forceinline__ T& E1(int r) { return e1[r]; }
  __device__ __forceinline__ T& D1(int r) { return d1[r]; }
  __device__ __forceinline__ T& E2(int r) { return e2[r]; }
  __device__ __forceinline__ T& D2(int r) { return d2[r]; }
};
template <int N>
__device__ __forceinline__ float& slot_of(float2 (&v)[N], int r) {
  return (r & 1) ? v[r >> 1].y : v[r >> 1].x;
}
template <int RPT>
struct Cols<float, RPT> {
  static_assert(RPT % 2 == 0, "FP32 ring slots come in pairs");
  static constexpr int NP = RPT / 2;
  float2 oh[NP], ol[NP], e1[NP], d1[NP], e2[NP], d2[NP];
  int k1[RPT], k2[RPT];
  __device__ __forceinline__ float& OH(int r) { return slot_of(oh, r); }
  __device__ __forceinline__ float& OL(int r) { return slot_of(ol, r); }
  __device__ __forceinline__ float& E1(int r) { return slot_of(e1, r); }
  __device__ __forceinline__ float& D1(int r) { return slot_of(d1, r); }
  __device__ __forceinline__ float& E2(int r) { return slot_of(e2, r); }
  __device__ __forceinline__ float& D2(int r) { return slot_of(d2, r); }
};

// synthesis sums of each slot: Re, Im of sum P e1, then of sum Q e2
template <typename T, int RPT>
struct SynAcc {
  T a[RPT][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < RPT; ++r) a[r][0] = a[r][1] = a[r][2] = a[r][3] = (T)0;
  }
  __device__ __forceinline__ T get(int r, int k) const { return a[r][k]; }
};
template <int RPT>
struct SynAcc<float, RPT> {
  float2 a[RPT / 2][4];  // slot pairs
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int p = 0; p < RPT / 2; ++p) a[p][0] = a[p][1] = a[p][2] = a[p][3] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float get(int r, int k) const { return (r & 1) ? a[r >> 1][k].y : a[r >> 1][k].x; }
};

// adjoint inputs of each slot: the ring values paired with column 1 (f1) and column 2 (f2)
template <typename T, int RPT>
struct AdjIn {
  using V = typename Cx<T>::V;
  V f1[RPT], f2[RPT];
  __device__ __forceinline__ void set(int r, V a, V b) {
    f1[r] = a;
    f2[r] = b;
  }
};
template <int RPT>
struct AdjIn<float, RPT> {
  float2 x1[RPT / 2], y1[RPT / 2], x2[RPT / 2], y2[RPT / 2];  // slot pairs of Re f1, Im f1, Re f2, Im f2
  __device__ __forceinline__ void set(int r, float2 a, float2 b) {
    slot_of(x1, r) = a.x;
    slot_of(y1, r) = a.y;
    slot_of(x2, r) = b.x;
    slot_of(y2, r) = b.y;
  }
};

// ---------------------------------------------------------------------------------------------
// one l step of a ring pair (FP32).  t = D - A (1 - x) with A, D and 1 - x as hi + lo:
//   t = (D_hi - A_hi oh) + ((D_lo - A_lo oh) - A_hi ol)
template <bool SPIN, int RPT>
__device__ __forceinline__ void step_pair(Cols<float, RPT>& S, int p, const TabEntry<float>& cf) {
  const float2 nah = lo2(cf.na), nal = hi2(cf.na);
  const float2 t = __fadd2_rn(__ffma2_rn(nah, S.oh[p], lo2(cf.d)),
                              __ffma2_rn(nah, S.ol[p], __ffma2_rn(nal, S.oh[p], hi2(cf.d))));
  const float2 B = lo2(cf.bc), C = hi2(cf.bc);
  if (SPIN) {
    reinsch_step2(__fadd2_rn(t, B), C, S.e1[p], S.d1[p]);
    reinsch_step2(__ffma2_rn(B, make_float2(-1.f, -1.f), t), C, S.e2[p], S.d2[p]);  // t - B
  } else {
    reinsch_step2(t, C, S.e1[p], S.d1[p]);
  }
}
// column values of a pair that take part in the sums: those with scale count 0
__device__ __forceinline__ float2 summing(float2 e, int ka, int kb) {
  return make_float2(ka == 0 ? e.x : 0.f, kb == 0 ? e.y : 0.f);
}

// One quad (4 l steps) of the synthesis for the ring slots r < nr of this thread, for NS sets of
// a_lm at once: the two Wigner columns of every (ring, l) are computed once and feed the sums of
// every set (P, Q of set k at sPQ[k * pqs + i]).  ACC: add the current column values to the sums;
// SEL: per column, only where k == 0.
template <bool SPIN, int RPT, bool ACC, bool SEL, bool TB, int NS>
__device__ __forceinline__ void syn_quad(Cols<double, RPT>& S, SynAcc<double, RPT> (&A)[NS],
                                         const TabEntry<double>* st, int i0, const Dbl4* sPQ, int pqs, int nr) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + u;
    const Coef cf = get_coef(st, i);
    Dbl4 pq[NS];
    if (ACC) {
#pragma unroll
      for (int k = 0; k < NS; ++k) pq[k] = sPQ[k * pqs + i];
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (r < nr) {
        if (ACC) {
          const double o1 = (!SEL || S.k1[r] == 0) ? S.e1[r] : 0.0;
          const double o2 = SPIN ? ((!SEL || S.k2[r] == 0) ? S.e2[r] : 0.0) : o1;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            A[k].a[r][0] = fma(pq[k].x, o1, A[k].a[r][0]);
            A[k].a[r][1] = fma(pq[k].y, o1, A[k].a[r][1]);
            A[k].a[r][2] = fma(pq[k].z, o2, A[k].a[r][2]);
            A[k].a[r][3] = fma(pq[k].w, o2, A[k].a[r][3]);
          }
        }
        col_steps<SPIN, TB>(cf, S.oh[r], S.e1[r], S.d1[r], S.e2[r], S.d2[r]);
      }
    }
  }
}
template <bool SPIN, int RPT, bool ACC, bool SEL, int NS>
__device__ __forceinline__ void syn_quad(Cols<float, RPT>& S, SynAcc<float, RPT> (&A)[NS], const TabEntry<float>* st,
                                         int i0, const PQ2* sPQ, int pqs, int nr) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + u;
    const TabEntry<float> cf = st[i];
    PQ2 pq[NS];
    if (ACC) {
#pragma unroll
      for (int k = 0; k < NS; ++k) pq[k] = sPQ[k * pqs + i];
    }
#pragma unroll
    for (int p = 0; p < RPT / 2; ++p) {
      if (2 * p < nr) {  // the second slot of the last pair may be empty: zero values, zero sums
        if (ACC) {
          const float2 o1 = SEL ? summing(S.e1[p], S.k1[2 * p], S.k1[2 * p + 1]) : S.e1[p];
          const float2 o2 = SPIN ? (SEL ? summing(S.e2[p], S.k2[2 * p], S.k2[2 * p + 1]) : S.e2[p]) : o1;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            A[k].a[p][0] = __ffma2_rn(lo2(pq[k].p), o1, A[k].a[p][0]);
            A[k].a[p][1] = __ffma2_rn(hi2(pq[k].p), o1, A[k].a[p][1]);
            A[k].a[p][2] = __ffma2_rn(lo2(pq[k].q), o2, A[k].a[p][2]);
            A[k].a[p][3] = __ffma2_rn(hi2(pq[k].q), o2, A[k].a[p][3]);
          }
        }
        step_pair<SPIN, RPT>(S, p, cf);
      }
    }
  }
}

// FP64 warps whose rings all lie at least kThreeTermDeg from the pole take the three-term form
// (tb); the FP32 form always takes Reinsch's
template <bool SPIN, int RPT, bool ACC, bool SEL, int NS, typename T, typename PQV>
__device__ __forceinline__ void syn_quad_d(bool tb, Cols<T, RPT>& S, SynAcc<T, RPT> (&A)[NS], const TabEntry<T>* st,
                                           int i0, const PQV* PQ, int pqs, int nr) {
  if constexpr (sizeof(T) == 8) {
    if (tb) syn_quad<SPIN, RPT, ACC, SEL, true, NS>(S, A, st, i0, PQ, pqs, nr);
    else syn_quad<SPIN, RPT, ACC, SEL, false, NS>(S, A, st, i0, PQ, pqs, nr);
  } else {
    syn_quad<SPIN, RPT, ACC, SEL, NS>(S, A, st, i0, PQ, pqs, nr);
  }
}

// decide the form of a warp's FP64 columns and convert them: oh <- x = 1 - (1 - x), and after
// init_col (fresh) d <- e_{l0-1} = 0 (slots >= nr are empty: zero columns).  Start states taken
// in the three-term form already hold e_{l-1} in d (fresh = false).
template <typename T, int RPT>
__device__ __forceinline__ bool three_term_setup(Cols<T, RPT>& S, int nr_slots, double omx_tb, bool fresh = true) {
  if constexpr (sizeof(T) == 8) {
    bool ok = true;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (r < nr_slots) ok = ok && S.OH(r) >= omx_tb;
    if (!__all_sync(0xffffffffu, ok)) return false;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      S.OH(r) = 1.0 - S.OH(r);
      if (fresh) {
        S.D1(r) = 0.0;
        S.D2(r) = 0.0;
      }
    }
    return true;
  } else {
    return false;
  }
}

template <typename T, bool SPIN, int RPT>
__device__ __forceinline__ void rescale_all(Cols<T, RPT>& S, int nr) {
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (r < nr) {
      rescale<T>(S.E1(r), S.D1(r), S.k1[r]);
      if (SPIN) rescale<T>(S.E2(r), S.D2(r), S.k2[r]);
    }
  }
}

// warp-uniform classification of the warp's columns: all summing / all still dropped.  vm: bit r
// set when slot r of this lane holds a ring; empty slots (zero values, zero counts) count as
// summing for the first test and are left out of the second, so that a part-filled warp still
// skips the sums while all of its rings are below the working range
template <typename T, bool SPIN, int RPT>
__device__ __forceinline__ void classify(const Cols<T, RPT>& S, int nr, unsigned vm, bool& fast, bool& skip) {
  bool in2 = true, in1 = true;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (r < nr) {
      in2 = in2 && S.k1[r] == 0 && S.k2[r] == 0;
      if ((vm >> r) & 1u) in1 = in1 && S.k1[r] > 0 && (!SPIN || S.k2[r] > 0);
    }
  }
  fast = __all_sync(0xffffffffu, in2);
  skip = !fast && __all_sync(0xffffffffu, in1);
}

// slots of this lane that hold rings (ring r * 32 + lane < n), as the bit mask classify takes
template <int RPT>
__device__ __forceinline__ unsigned slot_mask(int n, int lane) {
  unsigned vm = 0;
#pragma unroll
  for (int r = 0; r < RPT; ++r)
    if (r * 32 + lane < n) vm |= 1u << r;
  return vm;
}

// warp w of nw takes 32-ring slots [s0, s1) of the ceil(n/32) slots: first ring wbase, wcnt rings
__device__ __forceinline__ void slot_range(int n, int nw, int w, int& wbase, int& wcnt, int& nslot) {
  const int ns = (n + 31) >> 5;
  const int s0 = (w * ns) / nw, s1 = ((w + 1) * ns) / nw;
  wbase = 32 * s0;
  wcnt = max(0, min(32 * s1, n) - wbase);
  nslot = s1 - s0;
}

template <typename T, bool SPIN, int RPT>
__device__ __forceinline__ void init_col(Cols<T, RPT>& S, const RingDev* __restrict__ rings, const MSeed& sd,
                                         int jfirst, int jj, int nj, int r) {
  if (jj < nj) {
    const RingDev rg = rings[jfirst + jj];
    ring_omx<T>(rg, S.OH(r), S.OL(r));
    seed_scaled<T>(seed_log2(sd.lbin, sd.p1, sd.q1, rg.l2c, rg.l2s), sd.sign1, S.E1(r), S.k1[r]);
    if (SPIN) {
      seed_scaled<T>(seed_log2(sd.lbin, sd.q1, sd.p1, rg.l2c, rg.l2s), sd.sign2, S.E2(r), S.k2[r]);
    } else {
      S.E2(r) = (T)0;
      S.k2[r] = 0;
    }
  } else {
    // empty slot inside a partly filled warp: zero values that count as summing, so it adds
    // nothing and never holds the warp off the fast path
    S.OH(r) = S.OL(r) = S.E1(r) = S.E2(r) = (T)0;
    S.k1[r] = 0;
    S.k2[r] = 0;
  }
  S.D1(r) = S.E1(r);  // Delta_{l0} = e_{l0} - e_{l0-1}, e_{l0-1} = 0
  S.D2(r) = S.E2(r);
}

// Ring slots of a work item from the plan's start states (st, kk at the item's first slot): 1 - x
// from the ring table, the two columns, their differences (FP64 three-term form: e_{l-1}) and
// scale counts at the item's first working l (empty slots: zero values, zero counts, as init_col
// leaves them).  FP32 states are float4 (e1, d1, e2, d2), FP64 states four doubles.
template <typename T, bool SPIN, int RPT>
__device__ __forceinline__ void load_start(Cols<T, RPT>& S, const RingDev* __restrict__ rings, const void* st,
                                           const int* __restrict__ kk, int jfirst, int nj, int lane) {
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
    if (jj < nj) {
      ring_omx<T>(rings[jfirst + jj], S.OH(r), S.OL(r));
    } else {
      S.OH(r) = S.OL(r) = (T)0;
    }
    T e1, d1, e2, d2;
    if constexpr (sizeof(T) == 4) {
      const float4 v = reinterpret_cast<const float4*>(st)[jj];
      e1 = v.x, d1 = v.y, e2 = v.z, d2 = v.w;
    } else {
      const double2* q = reinterpret_cast<const double2*>(st) + 2 * jj;
      const double2 a = q[0], b = q[1];
      e1 = a.x, d1 = a.y, e2 = b.x, d2 = b.y;
    }
    const int k = kk[jj];
    S.E1(r) = e1;
    S.D1(r) = d1;
    S.E2(r) = SPIN ? e2 : (T)0;
    S.D2(r) = SPIN ? d2 : (T)0;
    S.k1[r] = k & 0xffff;
    S.k2[r] = SPIN ? (k >> 16) : 0;
  }
}

// ---------------------------------------------------------------------------------------------
// a_lm and ring-coefficient pointers of the NS sets of one synthesis launch (c may be null)
template <typename T, int NS>
struct SynSets {
  const typename Cx<T>::V* g[NS];
  const typename Cx<T>::V* c[NS];
  typename Cx<T>::V* F[NS];
};

// synthesis, one warp per CTA: the CTA's RecItem (order m, at most 32 RPT rings) is processed by a
// single warp, so there is no block barrier and a warp never waits for another warp's rings.  The
// warp stages its own table chunks of CH l (bulk copies issued by lane 0, NST stages in flight,
// completion on mbarriers) and its own P/Q values of every set (lane i computes l = lc + i, i < CH,
// from a_lm loaded one chunk ahead).  Ring slots: ring = r*32 + lane; slots r >= ceil(nj/32) are
// empty.  NS sets of a_lm share one pass over the table and one evaluation of the Wigner columns.
//
// MIR (mirror pairs, full-sky plans, NS = 1): the item's rings j (all at b <= pi/2) stand for the
// pairs (j, jm - j): ring jm - j lies at pi - b, where d^l_{m,-s}(pi - b) = (-1)^(l+m) d^l_{m,s}(b),
// so one evaluation of the two columns at b serves both.  The pair runs as two internal sets of
// the same a_lm: set 0 the direct ring, set 1 the mirror ring with the reflected combination of P
// and Q, written to ring jm - j.
template <typename T, bool SPIN, int RPT, int CH, int NST, int NS, bool MIR>
__global__ void __launch_bounds__(32) k_rec_syn_w(const RecItem* __restrict__ items, const RingDev* __restrict__ rings,
                                                  const MSeed* __restrict__ mseed, const TabEntry<T>* __restrict__ tab,
                                                  const SynSets<T, NS> sets, int lmax, int s, T msc, int Lpad,
                                                  int* __restrict__ status, double omx_tb, int jm,
                                                  const int* __restrict__ sls, const void* __restrict__ sst,
                                                  const int* __restrict__ skk) {
  static_assert(CH == 32, "one l per lane and chunk");
  static_assert(!MIR || NS == 1, "mirror pairs take one a_lm set");
  constexpr int NI = MIR ? 2 : NS;  // internal sets: the a_lm sets, or a ring and its mirror
  using V = typename Cx<T>::V;
  using PQV = typename PQRec<T>::V;
  const RecItem it = items[blockIdx.x];
  const int m = it.m;
  const MSeed sd = mseed[m];
  __shared__ __align__(16) TabStage<T, CH> stg[NST];
  __shared__ __align__(16) PQV sPQ[NI][NST][CH];
  __shared__ __align__(8) uint64_t bar[NST];
  constexpr int pqs = NST * CH;  // set stride of sPQ
  const int lane = threadIdx.x;
  const int nr_w = (it.nj + 31) >> 5;
  const unsigned vm = slot_mask<RPT>(it.nj, lane);
  Cols<T, RPT> S;
  SynAcc<T, RPT> A[NI];
#pragma unroll
  for (int k = 0; k < NI; ++k) A[k].zero();
  // first l of the recursion: the item's first working l, from the plan's start states (sls null:
  // l0, from the seeds)
  int lb = sd.l0;
  if (sls) {
    const int64_t so = (int64_t)blockIdx.x * RPT * 32;
    load_start<T, SPIN, RPT>(S, rings, (const unsigned char*)sst + so * 4 * sizeof(T), skk + so, it.j0, it.nj, lane);
    lb = sls[blockIdx.x];
  } else {
#pragma unroll
    for (int r = 0; r < RPT; ++r) init_col<T, SPIN, RPT>(S, rings, sd, it.j0, r * 32 + lane, it.nj, r);
  }
  // slots r with r * 32 + lane < nj hold rings
  const bool tb = three_term_setup<T, RPT>(S, lane < it.nj ? (it.nj - lane + 31) / 32 : 0, omx_tb, !sls);
  const int64_t base = alm_base(lmax, m);
  const bool rf = !MIR && it.refl != 0;
  const bool m0 = (m == 0);
  const int nchunk = max(0, (lmax - lb + CH) / CH);
  const V z = mk((T)0, (T)0);
  // internal set q: its a_lm set and whether its rings take the reflected combination
  const auto set_of = [&](int q) { return MIR ? 0 : q; };
  const auto refl_of = [&](int q) { return MIR ? (q == 1) : rf; };
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NST; ++k) mbar_init(&bar[k], 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (lane == 0)
    for (int k = 0; k < NST && k < nchunk; ++k) issue_chunk<T, CH>(stg[k], &bar[k], tab, base + lb + k * CH);
  for (int k = 0; k < NST && k < nchunk; ++k) {
    const int l = lb + k * CH + lane;
#pragma unroll
    for (int q = 0; q < NI; ++q) {
      V P = z, Q = z;
      const int qs = set_of(q);
      if (l <= lmax)
        make_pq<V, T>(sets.g[qs][base + l], sets.c[qs] ? sets.c[qs][base + l] : z, m0, refl_of(q), l + m, msc, P, Q);
      sPQ[q][k][lane] = pq_rec(P, Q);
    }
  }
  V pg[NS], pc[NS];  // a_lm of chunk NST (the next to be staged)
  {
    const int l = lb + NST * CH + lane;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      pg[q] = pc[q] = z;
      if (l <= lmax) {
        pg[q] = sets.g[q][base + l];
        if (sets.c[q]) pc[q] = sets.c[q][base + l];
      }
    }
  }
  __syncwarp();
  // once every column of the warp sums, it stays so (counts only fall, and only below the
  // working range): the warp then takes the plain path without testing its columns again
  bool fastw = false;

  for (int ch = 0; ch < nchunk; ++ch) {
    const int sidx = ch % NST;
    const bool ok = mbar_wait(&bar[sidx], (uint32_t)((ch / NST) & 1));
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) {
        atomicExch(status, 1);
        for (int k = ch + 1; k < nchunk && k < ch + NST; ++k)  // drain the copies still in flight
          mbar_wait(&bar[k % NST], (uint32_t)((k / NST) & 1));
      }
      return;
    }
    const int lc = lb + ch * CH;
    const int nq = (min(CH, lmax - lc + 1) + 3) >> 2;
    if (nr_w > 0) {
      const TabEntry<T>* st = stg[sidx].v;
      const PQV* PQ = &sPQ[0][sidx][0];
      for (int q = 0; q < nq; ++q) {
        bool fast = fastw, skip = false;
        if (!fastw) {
          classify<T, SPIN, RPT>(S, nr_w, vm, fast, skip);
          fastw = fast;
        }
        if (fast) {
          if (nr_w >= RPT) syn_quad_d<SPIN, RPT, true, false, NI>(tb, S, A, st, 4 * q, PQ, pqs, RPT);
          else syn_quad_d<SPIN, RPT, true, false, NI>(tb, S, A, st, 4 * q, PQ, pqs, nr_w);
        } else {
          if (skip) syn_quad_d<SPIN, RPT, false, false, NI>(tb, S, A, st, 4 * q, PQ, pqs, nr_w);
          else syn_quad_d<SPIN, RPT, true, true, NI>(tb, S, A, st, 4 * q, PQ, pqs, nr_w);
          rescale_all<T, SPIN, RPT>(S, nr_w);
        }
      }
    }
    __syncwarp();  // every lane is done with stage sidx
    if (ch + NST < nchunk) {
      if (lane == 0) issue_chunk<T, CH>(stg[sidx], &bar[sidx], tab, base + lc + NST * CH);
      const int l = lc + NST * CH + lane;
      const int l2 = l + CH;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        V P = z, Q = z;
        const int qs = set_of(q);
        if (l <= lmax) make_pq<V, T>(pg[qs], pc[qs], m0, refl_of(q), l + m, msc, P, Q);
        sPQ[q][sidx][lane] = pq_rec(P, Q);
      }
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        pg[q] = pc[q] = z;
        if (l2 <= lmax) {
          pg[q] = sets.g[q][base + l2];
          if (sets.c[q]) pc[q] = sets.c[q][base + l2];
        }
      }
    }
    __syncwarp();
  }
  const T sgn_s = (s & 1) ? (T)1 : (T)-1;  // -(-1)^s
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
    if (jj < it.nj) {
      const int j = it.j0 + jj;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        if (MIR && q == 1 && jm - j == j) continue;  // the equator ring is its own mirror
        const T a0 = A[q].get(r, 0), a1 = A[q].get(r, 1), a2 = A[q].get(r, 2), a3 = A[q].get(r, 3);
        const bool rq = refl_of(q);
        const V fpos = rq ? mk(-a2, -a3) : mk(-a0, -a1);
        const V fneg = rq ? mk(sgn_s * a0, sgn_s * a1) : mk(sgn_s * a2, sgn_s * a3);
        V* Fq = sets.F[set_of(q)];
        const int jq = (MIR && q == 1) ? jm - j : j;
        Fq[(int64_t)col_of(m) * Lpad + jq] = fpos;
        if (!m0) Fq[(int64_t)col_of(-m) * Lpad + jq] = fneg;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// adjoint: one CTA per order m (blockIdx.x = m), the active rings of one ring part, RPT rings per
// thread.  Per quad the 4 l values x 4 partial sums of each thread are reduced across the warp by
// a reduce-scatter (16 values over 32 lanes: 4 halving exchanges and one final add).
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

template <bool SPIN, int RPT, bool SEL, bool TB = false>
__device__ __forceinline__ void adj_quad_sums(Cols<double, RPT>& S, const AdjIn<double, RPT>& f,
                                              const TabEntry<double>* st, int i0, int nr, double (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const Coef cf = get_coef(st, i0 + u);
    double p0 = 0, p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (r < nr) {
        const double o1 = (!SEL || S.k1[r] == 0) ? S.e1[r] : 0.0;
        p0 = fma(o1, f.f1[r].x, p0);
        p1 = fma(o1, f.f1[r].y, p1);
        const double o2 = SPIN ? ((!SEL || S.k2[r] == 0) ? S.e2[r] : 0.0) : o1;
        p2 = fma(o2, f.f2[r].x, p2);
        p3 = fma(o2, f.f2[r].y, p3);
        col_steps<SPIN, TB>(cf, S.oh[r], S.e1[r], S.d1[r], S.e2[r], S.d2[r]);
      }
    }
    v[4 * u + 0] = p0;
    v[4 * u + 1] = p1;
    v[4 * u + 2] = p2;
    v[4 * u + 3] = p3;
  }
}
// mirror pairs (full-sky plans): sums of the direct rings against f plus (-1)^(l+m) times the
// column-swapped sums of their mirror rings against fm (reflected convention), lpm = l0 of the quad + m
template <bool SPIN, int RPT, bool SEL, bool TB>
__device__ __forceinline__ void adj_quad_sums_mir(Cols<double, RPT>& S, const AdjIn<double, RPT>& f,
                                                  const AdjIn<double, RPT>& fm, const TabEntry<double>* st, int i0,
                                                  int nr, int lpm, double (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const Coef cf = get_coef(st, i0 + u);
    double d0 = 0, d1 = 0, d2 = 0, d3 = 0, e0 = 0, e1 = 0, e2 = 0, e3 = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (r < nr) {
        const double o1 = (!SEL || S.k1[r] == 0) ? S.e1[r] : 0.0;
        const double o2 = SPIN ? ((!SEL || S.k2[r] == 0) ? S.e2[r] : 0.0) : o1;
        d0 = fma(o1, f.f1[r].x, d0);
        d1 = fma(o1, f.f1[r].y, d1);
        d2 = fma(o2, f.f2[r].x, d2);
        d3 = fma(o2, f.f2[r].y, d3);
        e0 = fma(o1, fm.f1[r].x, e0);
        e1 = fma(o1, fm.f1[r].y, e1);
        e2 = fma(o2, fm.f2[r].x, e2);
        e3 = fma(o2, fm.f2[r].y, e3);
        col_steps<SPIN, TB>(cf, S.oh[r], S.e1[r], S.d1[r], S.e2[r], S.d2[r]);
      }
    }
    const double sl = ((lpm + u) & 1) ? -1.0 : 1.0;
    v[4 * u + 0] = fma(sl, e2, d0);
    v[4 * u + 1] = fma(sl, e3, d1);
    v[4 * u + 2] = fma(sl, e0, d2);
    v[4 * u + 3] = fma(sl, e1, d3);
  }
}
template <bool SPIN, int RPT, bool SEL>
__device__ __forceinline__ void adj_quad_sums(Cols<float, RPT>& S, const AdjIn<float, RPT>& f,
                                              const TabEntry<float>* st, int i0, int nr, float (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const TabEntry<float> cf = st[i0 + u];
    float2 p0 = make_float2(0.f, 0.f), p1 = p0, p2 = p0, p3 = p0;  // (even slot, odd slot) partial sums
#pragma unroll
    for (int p = 0; p < RPT / 2; ++p) {
      if (2 * p < nr) {
        const float2 o1 = SEL ? summing(S.e1[p], S.k1[2 * p], S.k1[2 * p + 1]) : S.e1[p];
        p0 = __ffma2_rn(o1, f.x1[p], p0);
        p1 = __ffma2_rn(o1, f.y1[p], p1);
        const float2 o2 = SPIN ? (SEL ? summing(S.e2[p], S.k2[2 * p], S.k2[2 * p + 1]) : S.e2[p]) : o1;
        p2 = __ffma2_rn(o2, f.x2[p], p2);
        p3 = __ffma2_rn(o2, f.y2[p], p3);
        step_pair<SPIN, RPT>(S, p, cf);
      }
    }
    v[4 * u + 0] = p0.x + p0.y;
    v[4 * u + 1] = p1.x + p1.y;
    v[4 * u + 2] = p2.x + p2.y;
    v[4 * u + 3] = p3.x + p3.y;
  }
}
template <bool SPIN, int RPT, bool TB = false>
__device__ __forceinline__ void adj_quad_steps(Cols<double, RPT>& S, const TabEntry<double>* st, int i0, int nr) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const Coef cf = get_coef(st, i0 + u);
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (r < nr) col_steps<SPIN, TB>(cf, S.oh[r], S.e1[r], S.d1[r], S.e2[r], S.d2[r]);
  }
}
template <bool SPIN, int RPT>
__device__ __forceinline__ void adj_quad_steps(Cols<float, RPT>& S, const TabEntry<float>* st, int i0, int nr) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const TabEntry<float> cf = st[i0 + u];
#pragma unroll
    for (int p = 0; p < RPT / 2; ++p)
      if (2 * p < nr) step_pair<SPIN, RPT>(S, p, cf);
  }
}

// Start states of work items (plan time, one warp per item).  From the seeds at l0 the warp takes
// quads of 4 steps, with the arithmetic, the form (FP64: Reinsch's or the three-term one, decided
// as the kernels decide it) and the rescaling of the kernels' quads, while every column of its
// rings is still below the working range (empty slots do not count), and records the state at the
// first quad that has a working column.  Starting there, a kernel computes exactly what it would
// have computed from l0: the quads before it add nothing to any sum.  The quads read table records
// up to l + 3 <= lmax + 3, inside the table's zero padding.
template <typename T, bool SPIN, int RPT, typename Item>
__global__ void __launch_bounds__(32) k_rec_start(const Item* __restrict__ items, const RingDev* __restrict__ rings,
                                                  const MSeed* __restrict__ mseed, const TabEntry<T>* __restrict__ tab,
                                                  int lmax, double omx_tb, RecStart out) {
  const Item it = items[blockIdx.x];
  const int lane = threadIdx.x;
  const MSeed sd = mseed[it.m];
  const int nr_w = (it.nj + 31) >> 5;
  Cols<T, RPT> S;
#pragma unroll
  for (int r = 0; r < RPT; ++r) init_col<T, SPIN, RPT>(S, rings, sd, it.j0, r * 32 + lane, it.nj, r);
  const bool tb = three_term_setup<T, RPT>(S, lane < it.nj ? (it.nj - lane + 31) / 32 : 0, omx_tb);
  const TabEntry<T>* tv = tab + alm_base(lmax, it.m);
  int l = sd.l0;
  while (l <= lmax) {
    bool dropped = true;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (r < nr_w && r * 32 + lane < it.nj) dropped = dropped && S.k1[r] > 0 && (!SPIN || S.k2[r] > 0);
    if (!__all_sync(0xffffffffu, dropped)) break;
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const TabEntry<float> cf = tv[l + u];
#pragma unroll
        for (int p = 0; p < RPT / 2; ++p)
          if (2 * p < nr_w) step_pair<SPIN, RPT>(S, p, cf);
      }
    } else {
      if (tb) adj_quad_steps<SPIN, RPT, true>(S, tv, l, nr_w);
      else adj_quad_steps<SPIN, RPT, false>(S, tv, l, nr_w);
    }
    rescale_all<T, SPIN, RPT>(S, nr_w);
    l += 4;
  }
  if (lane == 0) out.ls[blockIdx.x] = l;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int64_t idx = ((int64_t)blockIdx.x * RPT + r) * 32 + lane;
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(out.st)[idx] = make_float4(S.E1(r), S.D1(r), S.E2(r), S.D2(r));
    } else {
      double2* q = reinterpret_cast<double2*>(out.st) + 2 * idx;
      q[0] = make_double2(S.E1(r), S.D1(r));
      q[1] = make_double2(S.E2(r), S.D2(r));
    }
    out.kk[idx] = S.k1[r] | (S.k2[r] << 16);
  }
}

// the three-term variants exist for FP64 only
template <bool SPIN, int RPT, bool SEL, bool TB, typename T>
__device__ __forceinline__ void adj_quad_sums_d(Cols<T, RPT>& S, const AdjIn<T, RPT>& f, const TabEntry<T>* st, int i0,
                                                int nr, T (&v)[16]) {
  if constexpr (sizeof(T) == 8) adj_quad_sums<SPIN, RPT, SEL, TB>(S, f, st, i0, nr, v);
  else adj_quad_sums<SPIN, RPT, SEL>(S, f, st, i0, nr, v);
}
template <bool SPIN, int RPT, bool TB, typename T>
__device__ __forceinline__ void adj_quad_steps_d(Cols<T, RPT>& S, const TabEntry<T>* st, int i0, int nr) {
  if constexpr (sizeof(T) == 8) adj_quad_steps<SPIN, RPT, TB>(S, st, i0, nr);
  else adj_quad_steps<SPIN, RPT>(S, st, i0, nr);
}

// Start states of the FP64 block adjoint (plan time): one CTA per order over the same rings and
// ring slots as k_rec_adj for one ring chunk of one ring part.  The CTA takes quads of 4 steps, as
// the kernel's warps take them while all their columns are dropped, as long as every column of
// every warp is still below the working range, and records the CTA's first working l (ls[m]) and
// each active ring's state there (at off[m] + the ring's index in the chunk).
template <bool SPIN, int RPT, int NT>
__global__ void __launch_bounds__(NT) k_rec_adj_start(const RingDev* __restrict__ rings,
                                                      const MSeed* __restrict__ mseed,
                                                      const int2* __restrict__ mrange,
                                                      const TabEntry<double>* __restrict__ tab, int lmax, int M,
                                                      int chunk, double omx_tb, const int64_t* __restrict__ off,
                                                      int* __restrict__ ls, double2* __restrict__ st,
                                                      int* __restrict__ kk) {
  const int m = blockIdx.x;
  if (m > M) return;
  const MSeed sd = mseed[m];
  int2 rr = mrange[m];
  rr.x += chunk * RPT * NT;
  rr.y = min(rr.y, rr.x + RPT * NT);
  const int nact = max(0, rr.y - rr.x);
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int wbase, wcnt, nr_w;
  slot_range(nact, NW, warp, wbase, wcnt, nr_w);
  Cols<double, RPT> S;
#pragma unroll
  for (int r = 0; r < RPT; ++r) init_col<double, SPIN, RPT>(S, rings, sd, rr.x + wbase, r * 32 + lane, wcnt, r);
  const bool tb = three_term_setup<double, RPT>(S, lane < wcnt ? (wcnt - lane + 31) / 32 : 0, omx_tb);
  const TabEntry<double>* tv = tab + alm_base(lmax, m);
  int l = sd.l0;
  while (nact > 0 && l <= lmax) {  // l and nact are the same in every thread of the CTA
    bool dropped = true;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (r < nr_w && r * 32 + lane < wcnt) dropped = dropped && S.k1[r] > 0 && (!SPIN || S.k2[r] > 0);
    if (!__syncthreads_and(dropped)) break;
    if (nr_w > 0) {
      if (tb) adj_quad_steps<SPIN, RPT, true>(S, tv, l, nr_w);
      else adj_quad_steps<SPIN, RPT, false>(S, tv, l, nr_w);
      rescale_all<double, SPIN, RPT>(S, nr_w);
    }
    l += 4;
  }
  if (threadIdx.x == 0) ls[m] = l;
  const int64_t o = off[m] + wbase;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
    if (jj < wcnt) {
      st[2 * (o + jj)] = make_double2(S.E1(r), S.D1(r));
      st[2 * (o + jj) + 1] = make_double2(S.E2(r), S.D2(r));
      kk[o + jj] = S.k1[r] | (S.k2[r] << 16);
    }
  }
}

// MIR: orders whose reflected rings are the mirrors jm - j of their direct rings (mmode[m] = 1,
// full-sky plans) run in the direct part's launches with both rings of each pair per slot; the
// launches of the other mode leave those orders alone (the first launch writes their zeros).
template <typename T, bool SPIN, int RPT, int NT, bool MIR>
__global__ void __launch_bounds__(NT) k_rec_adj(const RingDev* __restrict__ rings, const MSeed* __restrict__ mseed,
                                                const int2* __restrict__ mrange, const TabEntry<T>* __restrict__ tab,
                                                const typename Cx<T>::V* __restrict__ Ft, int Lpad,
                                                int lmax, int s, int M, int refl, int accumulate, T msc,
                                                typename Cx<T>::V* __restrict__ gt, typename Cx<T>::V* __restrict__ ct,
                                                int* __restrict__ status, int chunk, double omx_tb,
                                                const int* __restrict__ mmode, int jm,
                                                const int* __restrict__ sls, const int64_t* __restrict__ soff,
                                                const double2* __restrict__ sst, const int* __restrict__ skk) {
  using V = typename Cx<T>::V;
  const int m = blockIdx.x;
  const int64_t base = alm_base(lmax, m);
  if (m > M || (mmode && (m <= M) && ((mmode[m] != 0) != MIR))) {
    // beyond the polar-optimisation cutoff on every ring (transpose of a zero block), or an order
    // of the other mode: the first launch writes zeros, the others add nothing
    if (accumulate) return;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      gt[base + l] = mk((T)0, (T)0);
      if (ct) ct[base + l] = mk((T)0, (T)0);
    }
    return;
  }
  const MSeed sd = mseed[m];
  // rings of this launch: chunk `chunk` of RPT * NT rings of the part's active range
  int2 rr = mrange[m];
  rr.x += chunk * RPT * NT;
  rr.y = min(rr.y, rr.x + RPT * NT);
  if (rr.y <= rr.x) {
    if (accumulate) return;  // nothing to add
    rr.y = rr.x;             // first launch: write the zero projection below
  }
  const int nact = rr.y - rr.x;
  constexpr int NW = NT / 32;
  using V4 = typename Cx4<T>::V;  // 4 partial sums of one l
  __shared__ __align__(16) TabStage<T> stg[2];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int sfail;
  extern __shared__ __align__(16) unsigned char red_raw[];
  V4* red = reinterpret_cast<V4*>(red_raw);  // [2][NW][kCH]: double buffer of per-warp partial sums
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // first l: the CTA's first working l from the plan's start states (sls null: l0, from the seeds)
  const int lb = sls ? sls[m] : sd.l0;
  for (int l = m + threadIdx.x; !accumulate && l < lb && l <= lmax; l += blockDim.x) {
    gt[base + l] = mk((T)0, (T)0);
    if (ct) ct[base + l] = mk((T)0, (T)0);
  }
  const bool m0 = (m == 0);
  const bool rf = refl != 0;
  int wbase, wcnt, nr_w;  // ring slots as in the synthesis kernel
  slot_range(nact, NW, warp, wbase, wcnt, nr_w);

  Cols<T, RPT> S;
  AdjIn<T, RPT> fin;               // ring values paired with column 1 / column 2
  AdjIn<T, MIR ? RPT : 1> fmir;    // the mirror rings' values, reflected convention (MIR only)
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
    if (sls) {  // the ring's state at lb (empty slots: zero values and counts, as init_col leaves them)
      S.OH(r) = S.OL(r) = S.E1(r) = S.D1(r) = S.E2(r) = S.D2(r) = (T)0;
      S.k1[r] = S.k2[r] = 0;
      if (jj < wcnt) {
        ring_omx<T>(rings[rr.x + wbase + jj], S.OH(r), S.OL(r));
        const int64_t o = soff[m] + wbase + jj;
        const double2 a = sst[2 * o], b = sst[2 * o + 1];
        const int k = skk[o];
        S.E1(r) = (T)a.x;
        S.D1(r) = (T)a.y;
        if (SPIN) {
          S.E2(r) = (T)b.x;
          S.D2(r) = (T)b.y;
          S.k2[r] = k >> 16;
        }
        S.k1[r] = k & 0xffff;
      }
    } else {
      init_col<T, SPIN, RPT>(S, rings, sd, rr.x + wbase, jj, wcnt, r);
    }
    fin.set(r, mk((T)0, (T)0), mk((T)0, (T)0));
    if constexpr (MIR) {
      fmir.set(r, mk((T)0, (T)0), mk((T)0, (T)0));
      const int j = rr.x + wbase + jj;
      if (jj < wcnt && jm - j != j) {  // the equator ring is its own mirror
        const V fp = Ft[(int64_t)col_of(m) * Lpad + jm - j];
        const V fm = m0 ? mk((T)0, (T)0) : Ft[(int64_t)col_of(-m) * Lpad + jm - j];
        fmir.set(r, fm, fp);
      }
    }
    if (jj < wcnt) {
      const int j = rr.x + wbase + jj;
      const V fp = Ft[(int64_t)col_of(m) * Lpad + j];
      const V fm = m0 ? mk((T)0, (T)0) : Ft[(int64_t)col_of(-m) * Lpad + j];
      fin.set(r, rf ? fm : fp, rf ? fp : fm);
    }
  }
  const bool tb = three_term_setup<T, RPT>(S, lane < wcnt ? (wcnt - lane + 31) / 32 : 0, omx_tb, !sls);
  const unsigned vm = slot_mask<RPT>(wcnt, lane);
  const T sg = (((m - s) & 1) ? (T)1 : (T)-1);  // -(-1)^(m-s)
  const T sm = (m & 1) ? (T)-1 : (T)1;          // (-1)^m
  const int nchunk = max(0, (lmax - lb + kCH) / kCH);
  if (threadIdx.x == 0) {
    sfail = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (nchunk > 0) issue_chunk<T>(stg[0], &bar[0], tab, base + lb);
    if (nchunk > 1) issue_chunk<T>(stg[1], &bar[1], tab, base + lb + kCH);
  }

  for (int ch = 0; ch < nchunk; ++ch) {
    const int sidx = ch & 1;
    const int lc = lb + ch * kCH;
    const int n = min(kCH, lmax - lc + 1);
    const int nq = (n + 3) >> 2;
    if (!mbar_wait(&bar[sidx], (ch >> 1) & 1)) {
      atomicExch(status, 1);
      sfail = 1;
    }
    const TabEntry<T>* st = stg[sidx].v;
    T* redw = reinterpret_cast<T*>(red + (sidx * NW + warp) * kCH);
    for (int q = 0; q < nq; ++q) {
      T tot = (T)0;
      if (nr_w > 0 && !sfail) {
        bool fast, skip;
        classify<T, SPIN, RPT>(S, nr_w, vm, fast, skip);
        if (skip) {
          if (tb) adj_quad_steps_d<SPIN, RPT, true>(S, st, 4 * q, nr_w);
          else adj_quad_steps_d<SPIN, RPT, false>(S, st, 4 * q, nr_w);
          rescale_all<T, SPIN, RPT>(S, nr_w);
        } else {
          T v[16];
          if constexpr (MIR) {
            const int lpm = lc + 4 * q + m;
            if (fast) {
              if (tb) adj_quad_sums_mir<SPIN, RPT, false, true>(S, fin, fmir, st, 4 * q, nr_w, lpm, v);
              else adj_quad_sums_mir<SPIN, RPT, false, false>(S, fin, fmir, st, 4 * q, nr_w, lpm, v);
            } else {
              if (tb) adj_quad_sums_mir<SPIN, RPT, true, true>(S, fin, fmir, st, 4 * q, nr_w, lpm, v);
              else adj_quad_sums_mir<SPIN, RPT, true, false>(S, fin, fmir, st, 4 * q, nr_w, lpm, v);
              rescale_all<T, SPIN, RPT>(S, nr_w);
            }
          } else if (fast) {
            if (tb) {
              if (nr_w == RPT) adj_quad_sums_d<SPIN, RPT, false, true>(S, fin, st, 4 * q, RPT, v);
              else adj_quad_sums_d<SPIN, RPT, false, true>(S, fin, st, 4 * q, nr_w, v);
            } else {
              if (nr_w == RPT) adj_quad_sums_d<SPIN, RPT, false, false>(S, fin, st, 4 * q, RPT, v);
              else adj_quad_sums_d<SPIN, RPT, false, false>(S, fin, st, 4 * q, nr_w, v);
            }
          } else {
            if (tb) adj_quad_sums_d<SPIN, RPT, true, true>(S, fin, st, 4 * q, nr_w, v);
            else adj_quad_sums_d<SPIN, RPT, true, false>(S, fin, st, 4 * q, nr_w, v);
            rescale_all<T, SPIN, RPT>(S, nr_w);
          }
          tot = reduce_scatter16<T>(v, lane);
        }
      }
      if (lane < 16) redw[16 * q + lane] = tot;  // l = lc + 4q + (lane >> 2), sum (lane & 3)
    }
    __syncthreads();  // stage sidx consumed, partial sums of chunk ch complete
    if (sfail) {
      if (threadIdx.x == 0) mbar_wait(&bar[sidx ^ 1], ((ch + 1) >> 1) & 1);  // drain the other stage
      return;
    }
    if (ch + 2 < nchunk) {
      if (threadIdx.x == 0) issue_chunk<T>(stg[sidx], &bar[sidx], tab, base + lc + 2 * kCH);
    }
    for (int i = threadIdx.x; i < n; i += NT) {
      T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const V4 x = red[(sidx * NW + w) * kCH + i];
        q0 += x.x;
        q1 += x.y;
        q2 += x.z;
        q3 += x.w;
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
      if (!m0) {  // weight of the m > 0 entries (1, or 2 for the packed-gradient form; exact)
        gv = mk(msc * gv.x, msc * gv.y);
        cv = mk(msc * cv.x, msc * cv.y);
      }
      if (accumulate) {  // the projection is linear: the second ring part adds its share
        gv = cadd(gv, gt[id]);
        if (ct) cv = cadd(cv, ct[id]);
      }
      gt[id] = gv;
      if (ct) ct[id] = cv;
    }
    // no barrier here: the next chunk writes the other half of the double buffer, and the barrier
    // after it orders these reads before this half is written again
  }
}

// ---------------------------------------------------------------------------------------------
// adjoint, one warp per CTA (FP32 form): the warp's item is (m, up to 32 RPT rings), with the
// table staged as in k_rec_syn_w.  Per l each lane adds up its own rings' 4 products (Re, Im of
// the two columns) and stores them as one float4 row entry of a per-warp 8 x 32 shared array;
// after every 8 l (two quads) the warp sums the array's columns, lane i taking row i & 7 and a
// quarter of the columns (read swizzled so that no two lanes of an 8-lane phase share a bank
// group), then two shuffles combine the quarters: ~9 instructions per l and lane against ~20 for
// a shuffle reduce-scatter of the same sums.  The row totals (already in the direct-ring
// convention: reflected rings swap the column pairs and carry (-1)^(l+m)) then either
//   * go straight through the projection of the adjoint synthesis general formula to (g~, c~)
//     when the order m has a single item, or
//   * are added by one vector reduction (red.global.add.v4.f32) into the plan's accumulator of 4
//     floats per (l, m); the last item of m to finish (a per-m arrival counter) projects the
//     accumulated sums, writes (g~, c~) and clears the accumulator and the counter for the next
//     call.  The summation order of the reductions is not fixed, so for such orders the result
//     may differ between calls in the last bits.
// No block barrier and no waiting on other warps.  The projection:
//   ut_{l,m} = -Qp, ut_{l,-m} = -(-1)^(m-s) Qm, g~ = (ut_lm + (-1)^m conj ut_{l,-m})/2,
//   c~ = (ut_lm - (-1)^m conj ut_{l,-m})/(2i), zero below l0; msc weights m > 0 (1, or 2 in the
//   packed-gradient form).
__device__ __forceinline__ void adj_project(float4 q, bool m0, float sg, float sm, float msc, float2& gv,
                                            float2& cv) {
  const float ar = -q.x, ai = -q.y;
  const float br = sg * q.z, bi = sg * q.w;
  if (m0) {
    gv = make_float2(ar, 0.f);
    cv = make_float2(ai, 0.f);
  } else {
    const float wr = sm * br, wi = -sm * bi;  // (-1)^m conj(ut_{l,-m})
    gv = make_float2(msc * 0.5f * (ar + wr), msc * 0.5f * (ai + wi));
    cv = make_float2(msc * 0.5f * (ai - wi), msc * -0.5f * (ar - wr));
  }
}
__device__ __forceinline__ void red_add_v4(float4* addr, float4 v) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

// one quad (4 l steps) of the adjoint for the ring pairs of this thread and NS sets: per l the
// lane's sums over its rings (Re, Im against column 1; Re, Im against column 2) of set k go to row
// (row0 + u) of red[k]; the Wigner columns are evaluated once for all sets
template <bool SPIN, int RPT, bool SEL, int NS>
__device__ __forceinline__ void adj_quad_rows(Cols<float, RPT>& S, const AdjIn<float, RPT> (&f)[NS],
                                              const TabEntry<float>* st, int i0, int nr, float4 (*red)[8][32],
                                              int row0, int lane) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const TabEntry<float> cf = st[i0 + u];
    float2 p[NS][4];  // (even slot, odd slot) partial sums of each set
#pragma unroll
    for (int k = 0; k < NS; ++k) p[k][0] = p[k][1] = p[k][2] = p[k][3] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < RPT / 2; ++q) {
      if (2 * q < nr) {
        const float2 o1 = SEL ? summing(S.e1[q], S.k1[2 * q], S.k1[2 * q + 1]) : S.e1[q];
        const float2 o2 = SPIN ? (SEL ? summing(S.e2[q], S.k2[2 * q], S.k2[2 * q + 1]) : S.e2[q]) : o1;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          p[k][0] = __ffma2_rn(o1, f[k].x1[q], p[k][0]);
          p[k][1] = __ffma2_rn(o1, f[k].y1[q], p[k][1]);
          p[k][2] = __ffma2_rn(o2, f[k].x2[q], p[k][2]);
          p[k][3] = __ffma2_rn(o2, f[k].y2[q], p[k][3]);
        }
        step_pair<SPIN, RPT>(S, q, cf);
      }
    }
#pragma unroll
    for (int k = 0; k < NS; ++k)
      red[k][row0 + u][lane] =
          make_float4(p[k][0].x + p[k][0].y, p[k][1].x + p[k][1].y, p[k][2].x + p[k][2].y, p[k][3].x + p[k][3].y);
  }
}

// the same for mirror pairs (one set): the lane's direct rings give sums against F~_j (fd), their
// mirrors jm - j sums against F~_{jm-j} taken in the reflected convention (fm); per l the mirror
// part joins as (-1)^(l+m) times its column-swapped sums, so one row holds both
template <bool SPIN, int RPT, bool SEL>
__device__ __forceinline__ void adj_quad_rows_mir(Cols<float, RPT>& S, const AdjIn<float, RPT>& fd,
                                                  const AdjIn<float, RPT>& fm, const TabEntry<float>* st, int i0,
                                                  int nr, float4 (*red)[32], int row0, int lane, int lpm) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const TabEntry<float> cf = st[i0 + u];
    float2 d[4], e[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = e[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < RPT / 2; ++q) {
      if (2 * q < nr) {
        const float2 o1 = SEL ? summing(S.e1[q], S.k1[2 * q], S.k1[2 * q + 1]) : S.e1[q];
        const float2 o2 = SPIN ? (SEL ? summing(S.e2[q], S.k2[2 * q], S.k2[2 * q + 1]) : S.e2[q]) : o1;
        d[0] = __ffma2_rn(o1, fd.x1[q], d[0]);
        d[1] = __ffma2_rn(o1, fd.y1[q], d[1]);
        d[2] = __ffma2_rn(o2, fd.x2[q], d[2]);
        d[3] = __ffma2_rn(o2, fd.y2[q], d[3]);
        e[0] = __ffma2_rn(o1, fm.x1[q], e[0]);
        e[1] = __ffma2_rn(o1, fm.y1[q], e[1]);
        e[2] = __ffma2_rn(o2, fm.x2[q], e[2]);
        e[3] = __ffma2_rn(o2, fm.y2[q], e[3]);
        step_pair<SPIN, RPT>(S, q, cf);
      }
    }
    const float sl = ((lpm + u) & 1) ? -1.f : 1.f;  // (-1)^(l+m)
    red[row0 + u][lane] = make_float4(fmaf(sl, e[2].x + e[2].y, d[0].x + d[0].y),
                                      fmaf(sl, e[3].x + e[3].y, d[1].x + d[1].y),
                                      fmaf(sl, e[0].x + e[0].y, d[2].x + d[2].y),
                                      fmaf(sl, e[1].x + e[1].y, d[3].x + d[3].y));
  }
}

// ring coefficients in, accumulators and outputs of the NS sets of one adjoint launch (ct may be null)
template <int NS>
struct AdjSets {
  const float2* Ft[NS];
  float4* acc[NS];
  float2* gt[NS];
  float2* ct[NS];
};

// MIR (mirror pairs of full-sky plans, NS = 1): the item's rings j stand for the pairs (j, jm - j),
// whose two columns are shared (d^l_{m,-s}(pi - b) = (-1)^(l+m) d^l_{m,s}(b)); see adj_quad_rows_mir.
template <bool SPIN, int RPT, int CH, int NST, int NS, bool MIR>
__global__ void __launch_bounds__(32, NS == 1 ? (MIR ? 16 : (RPT >= 8 ? 16 : 20)) : (NS == 2 ? 12 : 8))
    k_rec_adj_w(const AdjItem* __restrict__ items, const RingDev* __restrict__ rings, const MSeed* __restrict__ mseed,
                const TabEntry<float>* __restrict__ tab, const AdjSets<NS> sets, int Lpad, int lmax, int s, float msc,
                int* __restrict__ cnt, int* __restrict__ status, int jm, const int* __restrict__ sls,
                const void* __restrict__ sst, const int* __restrict__ skk) {
  static_assert(CH % 8 == 0, "whole flushes of 8 l per chunk");
  static_assert(!MIR || NS == 1, "mirror pairs take one set");
  const AdjItem it = items[blockIdx.x];
  const int m = it.m;
  const MSeed sd = mseed[m];
  __shared__ __align__(16) TabStage<float, CH> stg[NST];
  __shared__ __align__(16) float4 red[NS][8][32];
  __shared__ __align__(8) uint64_t bar[NST];
  const int lane = threadIdx.x;
  const int nr_w = (it.nj + 31) >> 5;
  const unsigned vm = slot_mask<RPT>(it.nj, lane);
  const bool m0 = (m == 0);
  const bool rf = !MIR && it.refl != 0;
  const bool direct = it.nitems == 1;
  const float2 z = make_float2(0.f, 0.f);
  Cols<float, RPT> S;
  AdjIn<float, RPT> fin[NS];
  AdjIn<float, MIR ? RPT : 2> fmir;  // mirror rings' inputs in the reflected convention (MIR only)
  {  // columns at the item's first working l (plan start states)
    const int64_t so = (int64_t)blockIdx.x * RPT * 32;
    load_start<float, SPIN, RPT>(S, rings, reinterpret_cast<const float4*>(sst) + so, skk + so, it.j0, it.nj, lane);
  }
  const int lb = sls[blockIdx.x];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      fin[k].set(r, z, z);
      if (jj < it.nj) {
        const int j = it.j0 + jj;
        const float2 fp = sets.Ft[k][(int64_t)col_of(m) * Lpad + j];
        const float2 fm = m0 ? z : sets.Ft[k][(int64_t)col_of(-m) * Lpad + j];
        fin[k].set(r, rf ? fm : fp, rf ? fp : fm);
      }
    }
    if constexpr (MIR) {
      fmir.set(r, z, z);
      const int j = it.j0 + jj;
      if (jj < it.nj && jm - j != j) {  // the equator ring is its own mirror
        const float2 fp = sets.Ft[0][(int64_t)col_of(m) * Lpad + jm - j];
        const float2 fm = m0 ? z : sets.Ft[0][(int64_t)col_of(-m) * Lpad + jm - j];
        fmir.set(r, fm, fp);
      }
    }
  }
  const int64_t base = alm_base(lmax, m);
  const int nl = lmax - lb + 1;  // l = lb + li, li < nl (nl <= 0: no working column)
  const int nchunk = nl > 0 ? (nl + CH - 1) / CH : 0;
  const float sg = (((m - s) & 1) ? 1.f : -1.f);  // -(-1)^(m-s)
  const float sm = (m & 1) ? -1.f : 1.f;          // (-1)^m
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NST; ++k) mbar_init(&bar[k], 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (lane == 0)
    for (int k = 0; k < NST && k < nchunk; ++k) issue_chunk<float, CH>(stg[k], &bar[k], tab, base + lb + k * CH);
  __syncwarp();
  const int rr = lane & 7, cg = lane >> 3;  // flush: row and column quarter of this lane

  bool failed = false;
  bool blk_any = false;  // a quad of the current 8-l block had summing columns (warp-uniform)
  bool fastw = false;    // every column sums (then for good): no more column tests
  for (int ch = 0; ch < nchunk; ++ch) {
    const int sidx = ch % NST;
    const bool ok = mbar_wait(&bar[sidx], (uint32_t)((ch / NST) & 1));
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) {
        atomicExch(status, 1);
        for (int k = ch + 1; k < nchunk && k < ch + NST; ++k)  // drain the copies still in flight
          mbar_wait(&bar[k % NST], (uint32_t)((k / NST) & 1));
      }
      failed = true;
      break;
    }
    const int li0 = ch * CH;  // index of l = l0 + li0 in the order's l range
    const int nq = (min(CH, nl - li0) + 3) >> 2;
    const TabEntry<float>* st = stg[sidx].v;
    for (int q = 0; q < nq; ++q) {
      bool fast = fastw, skip = false;
      if (!fastw) {
        classify<float, SPIN, RPT>(S, nr_w, vm, fast, skip);
        fastw = fast;
      }
      blk_any = blk_any || !skip;
      const int row0 = (q & 1) * 4;
      if (skip) {
        adj_quad_steps<SPIN, RPT>(S, st, 4 * q, nr_w);
        rescale_all<float, SPIN, RPT>(S, nr_w);
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
          for (int u = 0; u < 4; ++u) red[k][row0 + u][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else if constexpr (MIR) {
        const int lpm = lb + li0 + 4 * q + m;
        if (fast) adj_quad_rows_mir<SPIN, RPT, false>(S, fin[0], fmir, st, 4 * q, nr_w, red[0], row0, lane, lpm);
        else {
          adj_quad_rows_mir<SPIN, RPT, true>(S, fin[0], fmir, st, 4 * q, nr_w, red[0], row0, lane, lpm);
          rescale_all<float, SPIN, RPT>(S, nr_w);
        }
      } else if (fast) {
        if (nr_w >= RPT) adj_quad_rows<SPIN, RPT, false, NS>(S, fin, st, 4 * q, RPT, red, row0, lane);
        else adj_quad_rows<SPIN, RPT, false, NS>(S, fin, st, 4 * q, nr_w, red, row0, lane);
      } else {
        adj_quad_rows<SPIN, RPT, true, NS>(S, fin, st, 4 * q, nr_w, red, row0, lane);
        rescale_all<float, SPIN, RPT>(S, nr_w);
      }
      if (((q & 1) || q == nq - 1) && !blk_any) {
        // every column of the block still below the working range: the sums are zero (single-item
        // orders write the zero projection, the others have nothing to add)
        const int li = li0 + 4 * (q & ~1) + lane;
        if (direct && lane < ((q & 1) ? 8 : 4) && li < nl) {
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            sets.gt[k][base + lb + li] = z;
            if (sets.ct[k]) sets.ct[k][base + lb + li] = z;
          }
        }
      } else if ((q & 1) || q == nq - 1) {  // flush rows 0 .. 8 (or 4) of red: l = l0 + li0 + 4 (q & ~1) + row
        blk_any = false;
        __syncwarp();
        const int li = li0 + 4 * (q & ~1) + lane;
        const bool out = lane < ((q & 1) ? 8 : 4) && li < nl;
        const int l = lb + li;
        const float sl = ((l + m) & 1) ? -1.f : 1.f;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const float4 x = red[k][rr][cg * 8 + (kk ^ rr)];
            a.x += x.x;
            a.y += x.y;
            a.z += x.z;
            a.w += x.w;
          }
#pragma unroll
          for (int o = 8; o <= 16; o <<= 1) {
            a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
            a.z += __shfl_xor_sync(0xffffffffu, a.z, o);
            a.w += __shfl_xor_sync(0xffffffffu, a.w, o);
          }
          if (out) {
            // sums against d_{m,-s}(theta) and d_{m,s}(theta): reflected rings swap the column
            // pairs and carry (-1)^(l+m)
            if (rf) a = make_float4(sl * a.z, sl * a.w, sl * a.x, sl * a.y);
            if (direct) {
              float2 gv, cv;
              adj_project(a, m0, sg, sm, msc, gv, cv);
              sets.gt[k][base + l] = gv;
              if (sets.ct[k]) sets.ct[k][base + l] = cv;
            } else {
              red_add_v4(&sets.acc[k][base + l], a);
            }
          }
        }
        __syncwarp();
      }
    }
    __syncwarp();  // every lane is done with stage sidx
    if (ch + NST < nchunk && lane == 0) issue_chunk<float, CH>(stg[sidx], &bar[sidx], tab, base + lb + (ch + NST) * CH);
    __syncwarp();
  }
  if (direct) {  // entries below the first working l (and below l0 for orders m < s) are zero
    for (int l = m + lane; l < lb && l <= lmax; l += 32) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        sets.gt[k][base + l] = z;
        if (sets.ct[k]) sets.ct[k][base + l] = z;
      }
    }
    return;
  }
  // arrival of this item; the last of the order's items projects the accumulated sums
  __threadfence();
  __syncwarp();
  int prev = 0;
  if (lane == 0) prev = atomicAdd(&cnt[m], 1);
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev != it.nitems - 1) return;
  __threadfence();
  for (int l = m + lane; l <= lmax; l += 32) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      float2 gv = z, cv = z;
      if (l >= sd.l0) {
        const float4 q = __ldcg(&sets.acc[k][base + l]);
        if (!failed) adj_project(q, m0, sg, sm, msc, gv, cv);
        __stcg(&sets.acc[k][base + l], make_float4(0.f, 0.f, 0.f, 0.f));
      }
      sets.gt[k][base + l] = gv;
      if (sets.ct[k]) sets.ct[k][base + l] = cv;
    }
  }
  if (lane == 0) cnt[m] = 0;
}

// orders without active rings (m > M) project to zero: (g~, c~) of orders [m_lo, m_hi)
template <typename V>
void zero_orders(const Plan& p, void* g, void* c, int m_lo, int m_hi, cudaStream_t st) {
  if (m_hi <= m_lo) return;
  // first packed index of order m: the orders m' < m hold lmax - m' + 1 entries each
  const auto off = [&](int m) { return (size_t)((int64_t)m * (2 * p.lmax + 3 - m) / 2); };
  const size_t b0 = off(m_lo) * sizeof(V), b1 = off(m_hi) * sizeof(V);
  PSHT_CUDA_TRY(cudaMemsetAsync((char*)g + b0, 0, b1 - b0, st));
  if (c) PSHT_CUDA_TRY(cudaMemsetAsync((char*)c + b0, 0, b1 - b0, st));
}

// one launch of the synthesis recursion for NS sets (items of the plan's current item range)
template <typename T, bool SPIN, int RPT, int NS>
void launch_syn_ns(Plan& p, const void* const* g, const void* const* c, void* const* F, double msc, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const int i0 = p.r_item0, i1 = p.r_item1 < 0 ? p.nitems : p.r_item1;
  SynSets<T, NS> ss;
  for (int k = 0; k < NS; ++k) {
    ss.g[k] = (const V*)g[k];
    ss.c[k] = c ? (const V*)c[k] : nullptr;
    ss.F[k] = (V*)F[k];
  }
  const int jm = p.nring - 1;
  // the items' start states, from the first item of the launch
  const int64_t so = (int64_t)i0 * RPT * 32;
  if (i1 > i0)
    k_rec_syn_w<T, SPIN, RPT, 32, 4, NS, false><<<i1 - i0, 32, 0, st>>>(
        p.d_items + i0, p.d_ring, p.d_mseed, (const TabEntry<T>*)p.d_rtab, ss, p.lmax, p.spin, (T)msc, p.Lpad,
        p.d_status, p.omx_tb, jm, p.s_items.ls + i0, (const unsigned char*)p.s_items.st + so * 4 * sizeof(T),
        p.s_items.kk + so);
  // mirror pairs of full-sky plans, one set at a time (they are never split into order chunks)
  if (p.nmitems > 0 && p.r_item1 < 0) {
    for (int k = 0; k < NS; ++k) {
      SynSets<T, 1> s1;
      s1.g[0] = ss.g[k];
      s1.c[0] = ss.c[k];
      s1.F[0] = ss.F[k];
      k_rec_syn_w<T, SPIN, RPT, 32, 4, 1, true><<<p.nmitems, 32, 0, st>>>(
          p.d_mitems, p.d_ring, p.d_mseed, (const TabEntry<T>*)p.d_rtab, s1, p.lmax, p.spin, (T)msc, p.Lpad,
          p.d_status, p.omx_tb, jm, p.s_mitems.ls, p.s_mitems.st, p.s_mitems.kk);
    }
  }
}
// nsets sets in launches of 4, 2 and 1 sets
template <typename T, bool SPIN, int RPT>
void launch_syn_t(Plan& p, int nsets, const void* const* g, const void* const* c, void* const* F, double msc,
                  cudaStream_t st) {
  for (int k = 0; k < nsets;) {
    const int left = nsets - k;
    const void* const* ck = c ? c + k : nullptr;
    if (left >= 4) {
      launch_syn_ns<T, SPIN, RPT, 4>(p, g + k, ck, F + k, msc, st);
      k += 4;
    } else if (left >= 2) {
      launch_syn_ns<T, SPIN, RPT, 2>(p, g + k, ck, F + k, msc, st);
      k += 2;
    } else {
      launch_syn_ns<T, SPIN, RPT, 1>(p, g + k, ck, F + k, msc, st);
      k += 1;
    }
  }
}

// one launch of the FP32 adjoint recursion for NS sets, then the zero orders of each set
template <bool SPIN, int RPT, int NS>
void launch_adj_ns(Plan& p, void* const* F, void* const* acc, void* const* g, void* const* c, double msc,
                   cudaStream_t st) {
  const int i0 = p.r_aitem0, i1 = p.r_aitem1 < 0 ? p.naitems : p.r_aitem1;
  const int m0 = p.r_m0, m1 = p.r_m1 < 0 ? p.lmax + 1 : p.r_m1;
  AdjSets<NS> as;
  for (int k = 0; k < NS; ++k) {
    as.Ft[k] = (const float2*)F[k];
    as.acc[k] = (float4*)acc[k];
    as.gt[k] = (float2*)g[k];
    as.ct[k] = c ? (float2*)c[k] : nullptr;
  }
  const int jm = p.nring - 1;
  const int64_t so = (int64_t)i0 * RPT * 32;
  if (i1 > i0)
    k_rec_adj_w<SPIN, RPT, 32, 4, NS, false><<<i1 - i0, 32, 0, st>>>(
        p.d_aitems + i0, p.d_ring, p.d_mseed, (const TabEntry<float>*)p.d_rtab, as, p.Lpad, p.lmax, p.spin,
        (float)msc, p.d_cnt, p.d_status, jm, p.s_aitems.ls + i0, reinterpret_cast<const float4*>(p.s_aitems.st) + so, p.s_aitems.kk + so);
  // mirror pairs of full-sky plans, one set at a time (never split into order chunks); their
  // orders' other items ran above, and the arrival counters join the two launches
  if (p.nmaitems > 0 && p.r_aitem1 < 0) {
    for (int k = 0; k < NS; ++k) {
      AdjSets<1> a1;
      a1.Ft[0] = as.Ft[k];
      a1.acc[0] = as.acc[k];
      a1.gt[0] = as.gt[k];
      a1.ct[0] = as.ct[k];
      k_rec_adj_w<SPIN, RPT, 32, 4, 1, true><<<p.nmaitems, 32, 0, st>>>(
          p.d_maitems, p.d_ring, p.d_mseed, (const TabEntry<float>*)p.d_rtab, a1, p.Lpad, p.lmax, p.spin, (float)msc,
          p.d_cnt, p.d_status, jm, p.s_maitems.ls, p.s_maitems.st, p.s_maitems.kk);
    }
  }
  for (int k = 0; k < NS; ++k) zero_orders<float2>(p, g[k], c ? c[k] : nullptr, std::max(m0, p.M + 1), m1, st);
}
template <bool SPIN, int RPT>
void launch_adj_w(Plan& p, int nsets, void* const* F, void* const* acc, void* const* g, void* const* c, double msc,
                  cudaStream_t st) {
  if (p.nmaitems > 0) {  // mirror pairs: the arrival counters count each item once per launch pair
    for (int k = 0; k < nsets; ++k)
      launch_adj_ns<SPIN, RPT, 1>(p, F + k, acc + k, g + k, c ? c + k : nullptr, msc, st);
    return;
  }
  for (int k = 0; k < nsets;) {
    const int left = nsets - k;
    void* const* ck = c ? c + k : nullptr;
    if (left >= 4) {
      launch_adj_ns<SPIN, RPT, 4>(p, F + k, acc + k, g + k, ck, msc, st);
      k += 4;
    } else if (left >= 2) {
      launch_adj_ns<SPIN, RPT, 2>(p, F + k, acc + k, g + k, ck, msc, st);
      k += 2;
    } else {
      launch_adj_ns<SPIN, RPT, 1>(p, F + k, acc + k, g + k, ck, msc, st);
      k += 1;
    }
  }
}

template <typename T, bool SPIN, int RPT, int NT>
void launch_adj_t(Plan& p, void* g, void* c, double msc, cudaStream_t st) {
  using V = typename Cx<T>::V;
  // one launch per ring part (rings at theta <= pi/2, then reflected rings at theta > pi/2) and
  // per chunk of RPT * NT rings of it; every launch after the first adds to the output
  const size_t red_bytes = (size_t)2 * (NT / 32) * kCH * sizeof(typename Cx4<T>::V);
  allow_dynamic_smem((const void*)k_rec_adj<T, SPIN, RPT, NT, false>, red_bytes);
  const int nch = (p.nring + RPT * NT - 1) / (RPT * NT);
  const int jm = p.nring - 1;
  const int2* mr0 = p.d_mrange;
  // start states of launch (part, chunk), if the plan has them
  const bool ss = p.s_badj.ls != nullptr && p.badj_nch == nch;
  const auto sls = [&](int part, int chk) { return ss ? p.s_badj.ls + (int64_t)(part * nch + chk) * (p.M + 1) : nullptr; };
  const auto soff = [&](int part, int chk) {
    return ss ? p.s_badj_off + (int64_t)(part * nch + chk) * (p.M + 1) : nullptr;
  };
  const double2* sst = ss ? (const double2*)p.s_badj.st : nullptr;
  const int* skk = ss ? p.s_badj.kk : nullptr;
  for (int part = 0; part < 2; ++part) {
    if (part == 1 && !p.has_refl) break;
    for (int chk = 0; chk < nch; ++chk)
      k_rec_adj<T, SPIN, RPT, NT, false><<<p.lmax + 1, NT, red_bytes, st>>>(
          p.d_ring, p.d_mseed, mr0 + part * (p.lmax + 1), (const TabEntry<T>*)p.d_rtab, (const V*)p.d_F,
          p.Lpad, p.lmax, p.spin, p.M, part, (part > 0 || chk > 0) ? 1 : 0, (T)msc, (V*)g, (V*)c, p.d_status, chk,
          p.omx_tb, p.d_mmode, jm, sls(part, chk), soff(part, chk), sst, skk);
    if (part == 0 && p.d_mmode) {  // mirror-pair orders of full-sky plans: direct rings with their mirrors
      allow_dynamic_smem((const void*)k_rec_adj<T, SPIN, RPT, NT, true>, red_bytes);
      for (int chk = 0; chk < nch; ++chk)
        k_rec_adj<T, SPIN, RPT, NT, true><<<p.lmax + 1, NT, red_bytes, st>>>(
            p.d_ring, p.d_mseed, mr0, (const TabEntry<T>*)p.d_rtab, (const V*)p.d_F, p.Lpad, p.lmax, p.spin, p.M, 0,
            1, (T)msc, (V*)g, (V*)c, p.d_status, chk, p.omx_tb, p.d_mmode, jm, sls(0, chk), soff(0, chk), sst, skk);
    }
  }
}

// FP64 block adjoint start states, one precompute launch per (ring part, ring chunk)
template <bool SPIN, int RPT, int NT>
void badj_starts_t(Plan& p, cudaStream_t st) {
  const int nch = (p.nring + RPT * NT - 1) / (RPT * NT);
  PSHT_REQUIRE(nch == p.badj_nch, PSHT_ECUDA, "internal: block adjoint chunks");
  for (int part = 0; part < (p.has_refl ? 2 : 1); ++part)
    for (int chk = 0; chk < nch; ++chk) {
      const int64_t o = (int64_t)(part * nch + chk) * (p.M + 1);
      k_rec_adj_start<SPIN, RPT, NT><<<p.M + 1, NT, 0, st>>>(
          p.d_ring, p.d_mseed, p.d_mrange + part * (p.lmax + 1), (const TabEntry<double>*)p.d_rtab, p.lmax, p.M, chk,
          p.omx_tb, p.s_badj_off + o, p.s_badj.ls + o, (double2*)p.s_badj.st, p.s_badj.kk);
    }
}
template <bool SPIN>
void badj_starts_s(Plan& p, cudaStream_t st) {
  switch (p.adj_rpt * 10000 + p.adj_threads) {
    case 20128: badj_starts_t<SPIN, 2, 128>(p, st); break;
    case 40128: badj_starts_t<SPIN, 4, 128>(p, st); break;
    case 40256: badj_starts_t<SPIN, 4, 256>(p, st); break;
    case 80128: badj_starts_t<SPIN, 8, 128>(p, st); break;
    case 80256: badj_starts_t<SPIN, 8, 256>(p, st); break;
    default: badj_starts_t<SPIN, 8, 512>(p, st); break;
  }
}

template <typename T, bool SPIN>
void launch_syn_s(Plan& p, int nsets, const void* const* g, const void* const* c, void* const* F, double msc,
                  cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    launch_syn_t<T, SPIN, 1>(p, nsets, g, c, F, msc, st);  // FP64: one ring per lane (syn_rpt 1)
  } else {
    launch_syn_t<T, SPIN, kSynRpt32>(p, nsets, g, c, F, msc, st);  // FP32: packed slot pairs
  }
}
template <typename T, bool SPIN>
void launch_adj_s(Plan& p, int nsets, void* const* F, void* const* acc, void* const* g, void* const* c, double msc,
                  cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {  // FP32: one warp per item, the sets in one launch
    launch_adj_w<SPIN, 4>(p, nsets, F, acc, g, c, msc, st);  // adj_rpt 4
    return;
  } else {
    // FP64 block form, one set at a time.  (rings per thread, threads) of one launch chunk are
    // chosen by the planner
    void* const F0 = p.d_F;
    for (int k = 0; k < nsets; ++k) {
      p.d_F = F[k];
      void* ck = c ? c[k] : nullptr;
      switch (p.adj_rpt * 10000 + p.adj_threads) {
        case 20128: launch_adj_t<T, SPIN, 2, 128>(p, g[k], ck, msc, st); break;
        case 40128: launch_adj_t<T, SPIN, 4, 128>(p, g[k], ck, msc, st); break;
        case 40256: launch_adj_t<T, SPIN, 4, 256>(p, g[k], ck, msc, st); break;
        case 80128: launch_adj_t<T, SPIN, 8, 128>(p, g[k], ck, msc, st); break;
        case 80256: launch_adj_t<T, SPIN, 8, 256>(p, g[k], ck, msc, st); break;
        default: launch_adj_t<T, SPIN, 8, 512>(p, g[k], ck, msc, st); break;
      }
    }
    p.d_F = F0;
  }
}

}  // namespace

int rec_table_record_bytes(int prec) {
  return prec == 64 ? (int)sizeof(TabEntry<double>) : (int)sizeof(TabEntry<float>);
}

void build_rec_table(Plan& p, cudaStream_t st) {
  const int nth = 128;
  const dim3 grid(p.lmax + 1, (p.lmax + 1 + nth - 1) / nth);  // blocks past lmax - m exit at once
  if (p.prec == 64) k_rec_table<double><<<grid, nth, 0, st>>>(p.lmax, p.spin, (TabEntry<double>*)p.d_rtab);
  else k_rec_table<float><<<grid, nth, 0, st>>>(p.lmax, p.spin, (TabEntry<float>*)p.d_rtab);
  PSHT_CUDA_TRY(cudaGetLastError());
}

void build_rec_starts(Plan& p, cudaStream_t st) {
  PSHT_REQUIRE(p.syn_threads == 32 && p.syn_rpt == (p.prec == 64 ? 1 : kSynRpt32), PSHT_ECUDA,
               "internal: synthesis shape");
  PSHT_REQUIRE(p.prec == 64 || (p.adj_rpt == 4 && p.adj_threads == 32), PSHT_ECUDA, "internal: FP32 adjoint shape");
  const auto run = [&](auto tag, auto spin) {
    using T = decltype(tag);
    constexpr bool S = decltype(spin)::value;
    constexpr int SR = sizeof(T) == 8 ? 1 : kSynRpt32;
    const auto* tab = (const TabEntry<T>*)p.d_rtab;
    if (p.nitems > 0)
      k_rec_start<T, S, SR, RecItem><<<p.nitems, 32, 0, st>>>(p.d_items, p.d_ring, p.d_mseed, tab, p.lmax, p.omx_tb,
                                                               p.s_items);
    if (p.nmitems > 0)
      k_rec_start<T, S, SR, RecItem><<<p.nmitems, 32, 0, st>>>(p.d_mitems, p.d_ring, p.d_mseed, tab, p.lmax,
                                                                p.omx_tb, p.s_mitems);
    if constexpr (sizeof(T) == 4) {
      if (p.naitems > 0)
        k_rec_start<float, S, 4, AdjItem><<<p.naitems, 32, 0, st>>>(p.d_aitems, p.d_ring, p.d_mseed, tab, p.lmax,
                                                                    p.omx_tb, p.s_aitems);
      if (p.nmaitems > 0)
        k_rec_start<float, S, 4, AdjItem><<<p.nmaitems, 32, 0, st>>>(p.d_maitems, p.d_ring, p.d_mseed, tab, p.lmax,
                                                                     p.omx_tb, p.s_maitems);
    }
  };
  if (p.prec == 64) {
    if (p.spin) run(0.0, std::true_type{});
    else run(0.0, std::false_type{});
    if (p.s_badj.ls) {
      if (p.spin) badj_starts_s<true>(p, st);
      else badj_starts_s<false>(p, st);
    }
  } else {
    if (p.spin) run(0.0f, std::true_type{});
    else run(0.0f, std::false_type{});
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_rec_synthesis_sets(Plan& p, int nsets, const void* const* g, const void* const* c, void* const* F,
                               cudaStream_t st, double msc) {
  if ((p.nitems == 0 && p.nmitems == 0) || nsets <= 0) return;  // full-sky plans may hold mirror items only
  if (p.prec == 64) {
    if (p.spin) launch_syn_s<double, true>(p, nsets, g, c, F, msc, st);
    else launch_syn_s<double, false>(p, nsets, g, c, F, msc, st);
  } else {
    if (p.spin) launch_syn_s<float, true>(p, nsets, g, c, F, msc, st);
    else launch_syn_s<float, false>(p, nsets, g, c, F, msc, st);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_rec_synthesis(Plan& p, const void* g, const void* c, cudaStream_t st, double msc) {
  void* F = p.d_F;
  launch_rec_synthesis_sets(p, 1, &g, c ? &c : nullptr, &F, st, msc);
}

void launch_rec_adjoint_sets(Plan& p, int nsets, void* const* F, void* const* acc, void* const* g, void* const* c,
                             cudaStream_t st, double msc) {
  if (nsets <= 0) return;
  if (p.prec == 64) {
    if (p.spin) launch_adj_s<double, true>(p, nsets, F, acc, g, c, msc, st);
    else launch_adj_s<double, false>(p, nsets, F, acc, g, c, msc, st);
  } else {
    if (p.spin) launch_adj_s<float, true>(p, nsets, F, acc, g, c, msc, st);
    else launch_adj_s<float, false>(p, nsets, F, acc, g, c, msc, st);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_rec_adjoint(Plan& p, void* g, void* c, cudaStream_t st, double msc) {
  void* F = p.d_F;
  void* acc = p.d_acc;
  launch_rec_adjoint_sets(p, 1, &F, &acc, &g, c ? &c : nullptr, st, msc);
}

}  // namespace psht
