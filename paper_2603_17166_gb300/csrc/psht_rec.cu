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
// working precision are carried as e 2^(-F k) and join the sums once k = 0.
//
// Synthesis (eq. syn on ring j):   F_j[m] = -sum_l (g + i c)_lm e1_l,   F_j[-m] = -(-1)^s sum_l (g* + i c*)_lm e2_l
// Adjoint (transpose, then the projection of the adjoint synthesis general formula, Sec. I):
//   ut_{l,m} = -sum_j e1_l(j) Ft_j[m],   ut_{l,-m} = -(-1)^(m-s) sum_j e2_l(j) Ft_j[-m]
//   g~ = (ut_lm + (-1)^m conj ut_{l,-m})/2,   c~ = (ut_lm - (-1)^m conj ut_{l,-m})/(2i)
//
// Data movement: per CTA the recurrence table of its order m is streamed through shared memory
// in chunks of 64 l by TMA bulk copies (cp.async.bulk, completion on an mbarrier, two stages in
// flight); the a_lm column is prefetched through registers two chunks ahead.
#include <cuda_runtime.h>
#include <math.h>

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

// One record of the recurrence table per packed (l, m), so that a chunk of 64 l is one contiguous
// bulk copy and one l is a few vector shared-memory loads.  The FP32 form works on pairs of rings
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

// One quad (4 l steps) of the synthesis for the ring slots r < nr of this thread.
// ACC: add the current column values to the sums; SEL: per column, only where k == 0.
template <bool SPIN, int RPT, bool ACC, bool SEL, bool TB = false>
__device__ __forceinline__ void syn_quad(Cols<double, RPT>& S, SynAcc<double, RPT>& A, const TabEntry<double>* st,
                                         int i0, const Dbl4* sPQ, int nr) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + u;
    const Coef cf = get_coef(st, i);
    const Dbl4 pq = sPQ[i];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (r < nr) {
        if (ACC) {
          const double o1 = (!SEL || S.k1[r] == 0) ? S.e1[r] : 0.0;
          A.a[r][0] = fma(pq.x, o1, A.a[r][0]);
          A.a[r][1] = fma(pq.y, o1, A.a[r][1]);
          const double o2 = SPIN ? ((!SEL || S.k2[r] == 0) ? S.e2[r] : 0.0) : o1;
          A.a[r][2] = fma(pq.z, o2, A.a[r][2]);
          A.a[r][3] = fma(pq.w, o2, A.a[r][3]);
        }
        col_steps<SPIN, TB>(cf, S.oh[r], S.e1[r], S.d1[r], S.e2[r], S.d2[r]);
      }
    }
  }
}
template <bool SPIN, int RPT, bool ACC, bool SEL>
__device__ __forceinline__ void syn_quad(Cols<float, RPT>& S, SynAcc<float, RPT>& A, const TabEntry<float>* st,
                                         int i0, const PQ2* sPQ, int nr) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + u;
    const TabEntry<float> cf = st[i];
    const PQ2 pq = sPQ[i];
#pragma unroll
    for (int p = 0; p < RPT / 2; ++p) {
      if (2 * p < nr) {  // the second slot of the last pair may be empty: zero values, zero sums
        if (ACC) {
          const float2 o1 = SEL ? summing(S.e1[p], S.k1[2 * p], S.k1[2 * p + 1]) : S.e1[p];
          A.a[p][0] = __ffma2_rn(lo2(pq.p), o1, A.a[p][0]);
          A.a[p][1] = __ffma2_rn(hi2(pq.p), o1, A.a[p][1]);
          const float2 o2 = SPIN ? (SEL ? summing(S.e2[p], S.k2[2 * p], S.k2[2 * p + 1]) : S.e2[p]) : o1;
          A.a[p][2] = __ffma2_rn(lo2(pq.q), o2, A.a[p][2]);
          A.a[p][3] = __ffma2_rn(hi2(pq.q), o2, A.a[p][3]);
        }
        step_pair<SPIN, RPT>(S, p, cf);
      }
    }
  }
}

// FP64 warps whose rings all lie at least kThreeTermDeg from the pole take the three-term form
// (tb); the FP32 form always takes Reinsch's
template <bool SPIN, int RPT, bool ACC, bool SEL, typename T, typename PQV>
__device__ __forceinline__ void syn_quad_d(bool tb, Cols<T, RPT>& S, SynAcc<T, RPT>& A, const TabEntry<T>* st, int i0,
                                           const PQV* PQ, int nr) {
  if constexpr (sizeof(T) == 8) {
    if (tb) {
      syn_quad<SPIN, RPT, ACC, SEL, true>(S, A, st, i0, PQ, nr);
      return;
    }
  }
  syn_quad<SPIN, RPT, ACC, SEL>(S, A, st, i0, PQ, nr);
}

// decide the form of a warp's FP64 columns after init_col and convert them: oh <- x = 1 - (1 - x),
// d <- e_{l0-1} = 0 (slots >= nr are empty: zero columns)
template <typename T, int RPT>
__device__ __forceinline__ bool three_term_setup(Cols<T, RPT>& S, int nr_slots, double omx_tb) {
  if constexpr (sizeof(T) == 8) {
    bool ok = true;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (r < nr_slots) ok = ok && S.OH(r) >= omx_tb;
    if (!__all_sync(0xffffffffu, ok)) return false;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      S.OH(r) = 1.0 - S.OH(r);
      S.D1(r) = 0.0;
      S.D2(r) = 0.0;
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

// warp-uniform classification of the warp's columns: all summing / all still dropped
template <typename T, bool SPIN, int RPT>
__device__ __forceinline__ void classify(const Cols<T, RPT>& S, int nr, bool& fast, bool& skip) {
  bool in2 = true, in1 = true;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (r < nr) {
      in2 = in2 && S.k1[r] == 0 && S.k2[r] == 0;
      in1 = in1 && S.k1[r] > 0 && (!SPIN || S.k2[r] > 0);
    }
  }
  fast = __all_sync(0xffffffffu, in2);
  skip = !fast && __all_sync(0xffffffffu, in1);
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

// ---------------------------------------------------------------------------------------------
// synthesis: one CTA of NT threads per RecItem (order m, rings j0 .. j0+nj-1), RPT rings per thread.
// Ring slots: warp w owns rings w*32*RPT + r*32 + lane (consecutive rings per warp, so the warp's
// columns leave the dropped region together); slots r >= nr_w are empty for the whole warp.
template <typename T, bool SPIN, int RPT, int NT>
__global__ void __launch_bounds__(NT) k_rec_syn(const RecItem* __restrict__ items, const RingDev* __restrict__ rings,
                                                const MSeed* __restrict__ mseed, const TabEntry<T>* __restrict__ tab,
                                                const typename Cx<T>::V* __restrict__ g,
                                                const typename Cx<T>::V* __restrict__ c, int lmax, int s, T msc,
                                                typename Cx<T>::V* __restrict__ F, int Lpad, int* __restrict__ status) {
  using V = typename Cx<T>::V;
  const RecItem it = items[blockIdx.x];
  const int m = it.m;
  const MSeed sd = mseed[m];
  __shared__ __align__(16) TabStage<T> stg[2];
  using PQV = typename PQRec<T>::V;
  __shared__ __align__(16) PQV sPQ[2][kCH];  // P and Q per l
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int sfail;

  // ring slots of 32 consecutive rings; the ceil(nj/32) slots are dealt to the warps in contiguous
  // runs differing by at most one, so a warp's columns leave the dropped region together and the
  // warps carry equal work; ring = wbase + r*32 + lane, slots r >= nr_w are empty for the warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int wbase, wcnt, nr_w;
  slot_range(it.nj, NT / 32, warp, wbase, wcnt, nr_w);
  Cols<T, RPT> S;
  SynAcc<T, RPT> A;
  A.zero();
#pragma unroll
  for (int r = 0; r < RPT; ++r) init_col<T, SPIN, RPT>(S, rings, sd, it.j0 + wbase, r * 32 + lane, wcnt, r);
  const int64_t base = alm_base(lmax, m);
  const bool rf = it.refl != 0;
  const bool m0 = (m == 0);
  const int nchunk = (lmax - sd.l0 + kCH) / kCH;

  // prologue: table chunks 0 and 1 by TMA, a_lm chunks 0 and 1 into shared memory, chunk 2 into
  // registers
  if (threadIdx.x == 0) {
    sfail = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    issue_chunk<T>(stg[0], &bar[0], tab, base + sd.l0);
    if (nchunk > 1) issue_chunk<T>(stg[1], &bar[1], tab, base + sd.l0 + kCH);
  }
  for (int cc = 0; cc < 2 && cc < nchunk; ++cc) {
    for (int i = threadIdx.x; i < kCH; i += NT) {
      const int l = sd.l0 + cc * kCH + i;
      V P = mk((T)0, (T)0), Q = mk((T)0, (T)0);
      if (l <= lmax) make_pq<V, T>(g[base + l], c ? c[base + l] : mk((T)0, (T)0), m0, rf, l + m, msc, P, Q);
      sPQ[cc][i] = pq_rec(P, Q);
    }
  }
  V pg = mk((T)0, (T)0), pc = mk((T)0, (T)0);  // a_lm two chunks ahead
  if (threadIdx.x < kCH) {
    const int l = sd.l0 + 2 * kCH + threadIdx.x;
    if (l <= lmax) {
      pg = g[base + l];
      if (c) pc = c[base + l];
    }
  }
  __syncthreads();

  for (int ch = 0; ch < nchunk; ++ch) {
    const int sidx = ch & 1;
    const int lc = sd.l0 + ch * kCH;
    if (!mbar_wait(&bar[sidx], (ch >> 1) & 1)) {
      atomicExch(status, 1);
      sfail = 1;
    }
    const int nq = (min(kCH, lmax - lc + 1) + 3) >> 2;
    if (nr_w > 0 && !sfail) {
      const TabEntry<T>* st = stg[sidx].v;
      const PQV* PQ = sPQ[sidx];
      for (int q = 0; q < nq; ++q) {
        bool fast, skip;
        classify<T, SPIN, RPT>(S, nr_w, fast, skip);
        if (fast) {
          if (nr_w == RPT) syn_quad<SPIN, RPT, true, false>(S, A, st, 4 * q, PQ, RPT);
          else syn_quad<SPIN, RPT, true, false>(S, A, st, 4 * q, PQ, nr_w);
        } else {
          if (skip) syn_quad<SPIN, RPT, false, false>(S, A, st, 4 * q, PQ, nr_w);
          else syn_quad<SPIN, RPT, true, true>(S, A, st, 4 * q, PQ, nr_w);
          rescale_all<T, SPIN, RPT>(S, nr_w);
        }
      }
    }
    __syncthreads();  // everyone is done with stage sidx
    if (sfail) {
      if (threadIdx.x == 0) mbar_wait(&bar[sidx ^ 1], ((ch + 1) >> 1) & 1);  // drain the other stage
      return;
    }
    if (ch + 2 < nchunk) {
      if (threadIdx.x == 0) issue_chunk<T>(stg[sidx], &bar[sidx], tab, base + lc + 2 * kCH);
      if (threadIdx.x < kCH) {
        const int l = lc + 2 * kCH + threadIdx.x;
        V Pn = mk((T)0, (T)0), Qn = mk((T)0, (T)0);
        if (l <= lmax) make_pq<V, T>(pg, pc, m0, rf, l + m, msc, Pn, Qn);
        sPQ[sidx][threadIdx.x] = pq_rec(Pn, Qn);
        pg = pc = mk((T)0, (T)0);
        const int l3 = l + kCH;
        if (l3 <= lmax) {
          pg = g[base + l3];
          if (c) pc = c[base + l3];
        }
      }
    }
  }
  const T sgn_s = (s & 1) ? (T)1 : (T)-1;  // -(-1)^s
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
    if (jj < wcnt) {
      const int j = it.j0 + wbase + jj;
      // direct rings: F[m] <- column 1, F[-m] <- column 2; reflected rings: swapped
      const T a0 = A.get(r, 0), a1 = A.get(r, 1), a2 = A.get(r, 2), a3 = A.get(r, 3);
      const V fpos = rf ? mk(-a2, -a3) : mk(-a0, -a1);
      const V fneg = rf ? mk(sgn_s * a0, sgn_s * a1) : mk(sgn_s * a2, sgn_s * a3);
      F[(int64_t)col_of(m) * Lpad + j] = fpos;
      if (!m0) F[(int64_t)col_of(-m) * Lpad + j] = fneg;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// synthesis, one warp per CTA: the CTA's RecItem (order m, at most 32 RPT rings) is processed by a
// single warp, so there is no block barrier and a warp never waits for another warp's rings.  The
// warp stages its own table chunks of CH l (bulk copies issued by lane 0, NST stages in flight,
// completion on mbarriers) and its own P/Q values (lane i computes l = lc + i, i < CH, from a_lm
// loaded one chunk ahead).  Ring slots: ring = r*32 + lane; slots r >= ceil(nj/32) are empty.
template <typename T, bool SPIN, int RPT, int CH, int NST>
__global__ void __launch_bounds__(32) k_rec_syn_w(const RecItem* __restrict__ items, const RingDev* __restrict__ rings,
                                                  const MSeed* __restrict__ mseed, const TabEntry<T>* __restrict__ tab,
                                                  const typename Cx<T>::V* __restrict__ g,
                                                  const typename Cx<T>::V* __restrict__ c, int lmax, int s, T msc,
                                                  typename Cx<T>::V* __restrict__ F, int Lpad,
                                                  int* __restrict__ status, double omx_tb) {
  static_assert(CH == 32, "one l per lane and chunk");
  using V = typename Cx<T>::V;
  using PQV = typename PQRec<T>::V;
  const RecItem it = items[blockIdx.x];
  const int m = it.m;
  const MSeed sd = mseed[m];
  __shared__ __align__(16) TabStage<T, CH> stg[NST];
  __shared__ __align__(16) PQV sPQ[NST][CH];
  __shared__ __align__(8) uint64_t bar[NST];
  const int lane = threadIdx.x;
  const int nr_w = (it.nj + 31) >> 5;
  Cols<T, RPT> S;
  SynAcc<T, RPT> A;
  A.zero();
#pragma unroll
  for (int r = 0; r < RPT; ++r) init_col<T, SPIN, RPT>(S, rings, sd, it.j0, r * 32 + lane, it.nj, r);
  // slots r with r * 32 + lane < nj hold rings
  const bool tb = three_term_setup<T, RPT>(S, lane < it.nj ? (it.nj - lane + 31) / 32 : 0, omx_tb);
  const int64_t base = alm_base(lmax, m);
  const bool rf = it.refl != 0;
  const bool m0 = (m == 0);
  const int nchunk = (lmax - sd.l0 + CH) / CH;
  const V z = mk((T)0, (T)0);

  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NST; ++k) mbar_init(&bar[k], 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (lane == 0)
    for (int k = 0; k < NST && k < nchunk; ++k) issue_chunk<T, CH>(stg[k], &bar[k], tab, base + sd.l0 + k * CH);
  for (int k = 0; k < NST && k < nchunk; ++k) {
    const int l = sd.l0 + k * CH + lane;
    V P = z, Q = z;
    if (l <= lmax) make_pq<V, T>(g[base + l], c ? c[base + l] : z, m0, rf, l + m, msc, P, Q);
    sPQ[k][lane] = pq_rec(P, Q);
  }
  V pg = z, pc = z;  // a_lm of chunk NST (the next to be staged)
  {
    const int l = sd.l0 + NST * CH + lane;
    if (l <= lmax) {
      pg = g[base + l];
      if (c) pc = c[base + l];
    }
  }
  __syncwarp();

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
    const int lc = sd.l0 + ch * CH;
    const int nq = (min(CH, lmax - lc + 1) + 3) >> 2;
    if (nr_w > 0) {
      const TabEntry<T>* st = stg[sidx].v;
      const PQV* PQ = sPQ[sidx];
      for (int q = 0; q < nq; ++q) {
        bool fast, skip;
        classify<T, SPIN, RPT>(S, nr_w, fast, skip);
        if (fast) {
          if (nr_w >= RPT) syn_quad_d<SPIN, RPT, true, false>(tb, S, A, st, 4 * q, PQ, RPT);
          else syn_quad_d<SPIN, RPT, true, false>(tb, S, A, st, 4 * q, PQ, nr_w);
        } else {
          if (skip) syn_quad_d<SPIN, RPT, false, false>(tb, S, A, st, 4 * q, PQ, nr_w);
          else syn_quad_d<SPIN, RPT, true, true>(tb, S, A, st, 4 * q, PQ, nr_w);
          rescale_all<T, SPIN, RPT>(S, nr_w);
        }
      }
    }
    __syncwarp();  // every lane is done with stage sidx
    if (ch + NST < nchunk) {
      if (lane == 0) issue_chunk<T, CH>(stg[sidx], &bar[sidx], tab, base + lc + NST * CH);
      const int l = lc + NST * CH + lane;
      V P = z, Q = z;
      if (l <= lmax) make_pq<V, T>(pg, pc, m0, rf, l + m, msc, P, Q);
      sPQ[sidx][lane] = pq_rec(P, Q);
      pg = pc = z;
      const int l2 = l + CH;
      if (l2 <= lmax) {
        pg = g[base + l2];
        if (c) pc = c[base + l2];
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
      const T a0 = A.get(r, 0), a1 = A.get(r, 1), a2 = A.get(r, 2), a3 = A.get(r, 3);
      const V fpos = rf ? mk(-a2, -a3) : mk(-a0, -a1);
      const V fneg = rf ? mk(sgn_s * a0, sgn_s * a1) : mk(sgn_s * a2, sgn_s * a3);
      F[(int64_t)col_of(m) * Lpad + j] = fpos;
      if (!m0) F[(int64_t)col_of(-m) * Lpad + j] = fneg;
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

template <typename T, bool SPIN, int RPT, int NT>
__global__ void __launch_bounds__(NT) k_rec_adj(const RingDev* __restrict__ rings, const MSeed* __restrict__ mseed,
                                                const int2* __restrict__ mrange, const TabEntry<T>* __restrict__ tab,
                                                const typename Cx<T>::V* __restrict__ Ft, int Lpad,
                                                int lmax, int s, int M, int refl, int accumulate, T msc,
                                                typename Cx<T>::V* __restrict__ gt, typename Cx<T>::V* __restrict__ ct,
                                                int* __restrict__ status, int chunk, double omx_tb) {
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
  for (int l = m + threadIdx.x; !accumulate && l < sd.l0 && l <= lmax; l += blockDim.x) {
    gt[base + l] = mk((T)0, (T)0);
    if (ct) ct[base + l] = mk((T)0, (T)0);
  }
  const bool m0 = (m == 0);
  const bool rf = refl != 0;
  int wbase, wcnt, nr_w;  // ring slots as in the synthesis kernel
  slot_range(nact, NW, warp, wbase, wcnt, nr_w);

  Cols<T, RPT> S;
  AdjIn<T, RPT> fin;  // ring values paired with column 1 / column 2
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
    init_col<T, SPIN, RPT>(S, rings, sd, rr.x + wbase, jj, wcnt, r);
    fin.set(r, mk((T)0, (T)0), mk((T)0, (T)0));
    if (jj < wcnt) {
      const int j = rr.x + wbase + jj;
      const V fp = Ft[(int64_t)col_of(m) * Lpad + j];
      const V fm = m0 ? mk((T)0, (T)0) : Ft[(int64_t)col_of(-m) * Lpad + j];
      fin.set(r, rf ? fm : fp, rf ? fp : fm);
    }
  }
  const bool tb = three_term_setup<T, RPT>(S, lane < wcnt ? (wcnt - lane + 31) / 32 : 0, omx_tb);
  const T sg = (((m - s) & 1) ? (T)1 : (T)-1);  // -(-1)^(m-s)
  const T sm = (m & 1) ? (T)-1 : (T)1;          // (-1)^m
  const int nchunk = (lmax - sd.l0 + kCH) / kCH;
  if (threadIdx.x == 0) {
    sfail = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    issue_chunk<T>(stg[0], &bar[0], tab, base + sd.l0);
    if (nchunk > 1) issue_chunk<T>(stg[1], &bar[1], tab, base + sd.l0 + kCH);
  }

  for (int ch = 0; ch < nchunk; ++ch) {
    const int sidx = ch & 1;
    const int lc = sd.l0 + ch * kCH;
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
        classify<T, SPIN, RPT>(S, nr_w, fast, skip);
        if (skip) {
          if (tb) adj_quad_steps_d<SPIN, RPT, true>(S, st, 4 * q, nr_w);
          else adj_quad_steps_d<SPIN, RPT, false>(S, st, 4 * q, nr_w);
          rescale_all<T, SPIN, RPT>(S, nr_w);
        } else {
          T v[16];
          if (fast) {
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
// table staged as in k_rec_syn_w.  Per quad of l the warp's 16 partial sums are reduced across
// the lanes (reduce_scatter16) and written to the item's slice of the partial-sum array, already
// in the direct-ring convention (reflected rings: columns swapped, signed by (-1)^(l+m)); the
// items of one m are then summed and projected by k_adj_reduce.  No block barrier, no atomics,
// and the result does not depend on scheduling.
template <typename T, bool SPIN, int RPT, int CH, int NST>
__global__ void __launch_bounds__(32) k_rec_adj_w(const AdjItem* __restrict__ items, const RingDev* __restrict__ rings,
                                                  const MSeed* __restrict__ mseed, const TabEntry<T>* __restrict__ tab,
                                                  const typename Cx<T>::V* __restrict__ Ft, int Lpad, int lmax,
                                                  T* __restrict__ part, int* __restrict__ status) {
  static_assert(CH % 4 == 0, "whole quads per chunk");
  using V = typename Cx<T>::V;
  const AdjItem it = items[blockIdx.x];
  const int m = it.m;
  const MSeed sd = mseed[m];
  __shared__ __align__(16) TabStage<T, CH> stg[NST];
  __shared__ __align__(8) uint64_t bar[NST];
  const int lane = threadIdx.x;
  const int nr_w = (it.nj + 31) >> 5;
  const bool m0 = (m == 0);
  const bool rf = it.refl != 0;
  const V z = mk((T)0, (T)0);
  Cols<T, RPT> S;
  AdjIn<T, RPT> fin;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int jj = r * 32 + lane;
    init_col<T, SPIN, RPT>(S, rings, sd, it.j0, jj, it.nj, r);
    fin.set(r, z, z);
    if (jj < it.nj) {
      const int j = it.j0 + jj;
      const V fp = Ft[(int64_t)col_of(m) * Lpad + j];
      const V fm = m0 ? z : Ft[(int64_t)col_of(-m) * Lpad + j];
      fin.set(r, rf ? fm : fp, rf ? fp : fm);
    }
  }
  const int64_t base = alm_base(lmax, m);
  const int nl = lmax - sd.l0 + 1;
  const int nchunk = (nl + CH - 1) / CH;
  T* out = part + it.off;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NST; ++k) mbar_init(&bar[k], 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (lane == 0)
    for (int k = 0; k < NST && k < nchunk; ++k) issue_chunk<T, CH>(stg[k], &bar[k], tab, base + sd.l0 + k * CH);
  __syncwarp();

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
    const int li0 = ch * CH;  // index of l = l0 + li0 in the item's slice
    const int nq = (min(CH, nl - li0) + 3) >> 2;
    const TabEntry<T>* st = stg[sidx].v;
    for (int q = 0; q < nq; ++q) {
      T tot = (T)0;
      bool fast, skip;
      classify<T, SPIN, RPT>(S, nr_w, fast, skip);
      if (skip) {
        adj_quad_steps<SPIN, RPT>(S, st, 4 * q, nr_w);
        rescale_all<T, SPIN, RPT>(S, nr_w);
      } else {
        T v[16];
        if (fast) {
          if (nr_w >= RPT) adj_quad_sums<SPIN, RPT, false>(S, fin, st, 4 * q, RPT, v);
          else adj_quad_sums<SPIN, RPT, false>(S, fin, st, 4 * q, nr_w, v);
        } else {
          adj_quad_sums<SPIN, RPT, true>(S, fin, st, 4 * q, nr_w, v);
          rescale_all<T, SPIN, RPT>(S, nr_w);
        }
        tot = reduce_scatter16<T>(v, lane);  // lane < 16: sum (lane & 3) of l = 4q + (lane >> 2)
      }
      const int li = li0 + 4 * q + ((lane >> 2) & 3);
      if (rf) {  // sums against d_{m,-s}(theta) and d_{m,s}(theta): swap the column pairs, sign (-1)^(l+m)
        const T other = __shfl_xor_sync(0xffffffffu, tot, 2);
        tot = (((sd.l0 + li + m) & 1) ? (T)-1 : (T)1) * other;
      }
      if (lane < 16 && li < nl) out[4 * (int64_t)li + (lane & 3)] = tot;
    }
    __syncwarp();  // every lane is done with stage sidx
    if (ch + NST < nchunk && lane == 0) issue_chunk<T, CH>(stg[sidx], &bar[sidx], tab, base + sd.l0 + (ch + NST) * CH);
    __syncwarp();
  }
}

// Sum of the adjoint items of order m (m_first + blockIdx.x) and the projection of the adjoint synthesis
// general formula: ut_{l,m} = -Qp, ut_{l,-m} = -(-1)^(m-s) Qm, g~ = (ut_lm + (-1)^m conj ut_{l,-m})/2,
// c~ = (ut_lm - (-1)^m conj ut_{l,-m})/(2i); zero below l0 and for orders without active rings.
template <typename T>
__global__ void k_adj_reduce(const AdjItem* __restrict__ items, const int2* __restrict__ aspan,
                             const MSeed* __restrict__ mseed, const T* __restrict__ part, int lmax, int s, T msc,
                             int m_first, typename Cx<T>::V* __restrict__ gt, typename Cx<T>::V* __restrict__ ct) {
  using V = typename Cx<T>::V;
  constexpr int kMaxItems = 64;
  __shared__ int64_t off[kMaxItems];
  const int m = m_first + blockIdx.x;
  const int2 sp = aspan[m];
  const int64_t base = alm_base(lmax, m);
  const int l0 = sp.y > 0 ? mseed[m].l0 : lmax + 1;
  for (int k = threadIdx.x; k < sp.y && k < kMaxItems; k += blockDim.x) off[k] = items[sp.x + k].off;
  __syncthreads();
  const bool m0 = (m == 0);
  const T sg = (((m - s) & 1) ? (T)1 : (T)-1);  // -(-1)^(m-s)
  const T sm = (m & 1) ? (T)-1 : (T)1;          // (-1)^m
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    V gv = mk((T)0, (T)0), cv = gv;
    if (l >= l0) {
      T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
      const int64_t li = 4 * (int64_t)(l - l0);
      for (int k = 0; k < sp.y; ++k) {
        const int64_t o = (k < kMaxItems ? off[k] : items[sp.x + k].off) + li;
        q0 += part[o];
        q1 += part[o + 1];
        q2 += part[o + 2];
        q3 += part[o + 3];
      }
      const T ar = -q0, ai = -q1;
      const T br = sg * q2, bi = sg * q3;
      if (m0) {
        gv = mk(ar, (T)0);
        cv = mk(ai, (T)0);
      } else {
        const T wr = sm * br, wi = -sm * bi;  // (-1)^m conj(ut_{l,-m})
        gv = mk(msc * (T)0.5 * (ar + wr), msc * (T)0.5 * (ai + wi));
        cv = mk(msc * (T)0.5 * (ai - wi), msc * (T)-0.5 * (ar - wr));
      }
    }
    gt[base + l] = gv;
    if (ct) ct[base + l] = cv;
  }
}

template <typename T, bool SPIN, int RPT>
void launch_syn_t(Plan& p, const void* g, const void* c, double msc, cudaStream_t st) {
  using V = typename Cx<T>::V;
  if (p.syn_threads == 32) {  // one warp per item (items of at most 32 RPT rings)
    const int i0 = p.r_item0, i1 = p.r_item1 < 0 ? p.nitems : p.r_item1;
    if (i1 > i0)
      k_rec_syn_w<T, SPIN, RPT, 32, 4><<<i1 - i0, 32, 0, st>>>(
          p.d_items + i0, p.d_ring, p.d_mseed, (const TabEntry<T>*)p.d_rtab, (const V*)g, (const V*)c, p.lmax,
          p.spin, (T)msc, (V*)p.d_F, p.Lpad, p.d_status, p.omx_tb);
    return;
  }
  k_rec_syn<T, SPIN, RPT, 128><<<p.nitems, 128, 0, st>>>(p.d_items, p.d_ring, p.d_mseed,
                                                          (const TabEntry<T>*)p.d_rtab, (const V*)g, (const V*)c, p.lmax, p.spin, (T)msc,
                                                          (V*)p.d_F, p.Lpad, p.d_status);
}

template <typename T, bool SPIN, int RPT>
void launch_adj_w(Plan& p, void* g, void* c, double msc, cudaStream_t st) {
  using V = typename Cx<T>::V;
  const int i0 = p.r_aitem0, i1 = p.r_aitem1 < 0 ? p.naitems : p.r_aitem1;
  const int m0 = p.r_m0, m1 = p.r_m1 < 0 ? p.lmax + 1 : p.r_m1;
  if (i1 > i0)
    k_rec_adj_w<T, SPIN, RPT, 32, 4><<<i1 - i0, 32, 0, st>>>(p.d_aitems + i0, p.d_ring, p.d_mseed,
                                                              (const TabEntry<T>*)p.d_rtab, (const V*)p.d_F, p.Lpad,
                                                              p.lmax, (T*)p.d_part, p.d_status);
  if (m1 > m0)
    k_adj_reduce<T><<<m1 - m0, 256, 0, st>>>(p.d_aitems, p.d_aspan, p.d_mseed, (const T*)p.d_part, p.lmax, p.spin,
                                             (T)msc, m0, (V*)g, (V*)c);
}

template <typename T, bool SPIN, int RPT, int NT>
void launch_adj_t(Plan& p, void* g, void* c, double msc, cudaStream_t st) {
  using V = typename Cx<T>::V;
  // one launch per ring part (rings at theta <= pi/2, then reflected rings at theta > pi/2) and
  // per chunk of RPT * NT rings of it; every launch after the first adds to the output
  const size_t red_bytes = (size_t)2 * (NT / 32) * kCH * sizeof(typename Cx4<T>::V);
  PSHT_CUDA_TRY(cudaFuncSetAttribute((const void*)k_rec_adj<T, SPIN, RPT, NT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red_bytes));
  const int nch = (p.nring + RPT * NT - 1) / (RPT * NT);
  for (int part = 0; part < 2; ++part) {
    if (part == 1 && !p.has_refl) break;
    for (int chk = 0; chk < nch; ++chk)
      k_rec_adj<T, SPIN, RPT, NT><<<p.lmax + 1, NT, red_bytes, st>>>(
          p.d_ring, p.d_mseed, p.d_mrange + part * (p.lmax + 1), (const TabEntry<T>*)p.d_rtab, (const V*)p.d_F,
          p.Lpad, p.lmax, p.spin, p.M, part, (part > 0 || chk > 0) ? 1 : 0, (T)msc, (V*)g, (V*)c, p.d_status, chk,
          p.omx_tb);
  }
}

template <typename T, bool SPIN>
void launch_syn_s(Plan& p, const void* g, const void* c, double msc, cudaStream_t st) {
  switch (p.syn_rpt) {
    case 1: launch_syn_t<T, SPIN, sizeof(T) == 8 ? 1 : 2>(p, g, c, msc, st); break;  // FP32 slots come in pairs
    case 2: launch_syn_t<T, SPIN, 2>(p, g, c, msc, st); break;
    default: launch_syn_t<T, SPIN, 4>(p, g, c, msc, st); break;
  }
}
template <typename T, bool SPIN>
void launch_adj_s(Plan& p, void* g, void* c, double msc, cudaStream_t st) {
  if (p.adj_threads == 32) {  // one warp per item, FP32 form
    if constexpr (sizeof(T) == 4) {
      if (p.adj_rpt == 8) launch_adj_w<T, SPIN, 8>(p, g, c, msc, st);
      else if (p.adj_rpt == 2) launch_adj_w<T, SPIN, 2>(p, g, c, msc, st);
      else launch_adj_w<T, SPIN, 4>(p, g, c, msc, st);
      return;
    }
  }
  // (rings per thread, threads) of one launch chunk; chosen by the planner
  switch (p.adj_rpt * 10000 + p.adj_threads) {
    case 20128: launch_adj_t<T, SPIN, 2, 128>(p, g, c, msc, st); break;
    case 40128: launch_adj_t<T, SPIN, 4, 128>(p, g, c, msc, st); break;
    case 40256: launch_adj_t<T, SPIN, 4, 256>(p, g, c, msc, st); break;
    case 80128: launch_adj_t<T, SPIN, 8, 128>(p, g, c, msc, st); break;
    case 80256: launch_adj_t<T, SPIN, 8, 256>(p, g, c, msc, st); break;
    default: launch_adj_t<T, SPIN, 8, 512>(p, g, c, msc, st); break;
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

void launch_rec_synthesis(Plan& p, const void* g, const void* c, cudaStream_t st, double msc) {
  if (p.nitems == 0) return;
  if (p.prec == 64) {
    if (p.spin) launch_syn_s<double, true>(p, g, c, msc, st);
    else launch_syn_s<double, false>(p, g, c, msc, st);
  } else {
    if (p.spin) launch_syn_s<float, true>(p, g, c, msc, st);
    else launch_syn_s<float, false>(p, g, c, msc, st);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

void launch_rec_adjoint(Plan& p, void* g, void* c, cudaStream_t st, double msc) {
  if (p.prec == 64) {
    if (p.spin) launch_adj_s<double, true>(p, g, c, msc, st);
    else launch_adj_s<double, false>(p, g, c, msc, st);
  } else {
    if (p.spin) launch_adj_s<float, true>(p, g, c, msc, st);
    else launch_adj_s<float, false>(p, g, c, msc, st);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

}  // namespace psht
