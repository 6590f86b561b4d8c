// Change of frame: Wigner-D rotation of a_lm sets, rotation of points with the spin-basis angle,
// and the patch-centred frame (smallest cap around the points).
//
// The paper evaluates its rings about a pole placed at the patch centre (Sec. II, step 1).  To let
// a caller keep a_lm and points in their own frame, the coefficients are rotated with
//   a'_lm = sum_m' e^{-i m alpha} d^l_{m m'}(beta) e^{-i m' gamma} a_lm'
// and d^l(beta) is factorised through Delta^l = d^l(pi/2) by the appendix's Fourier identity
//   d^l_{m m'}(beta) = sum_k i^m Delta_{k m} e^{-i k beta} Delta_{k m'} (-i)^m'.
// A rotation is then two contractions with Delta^l per degree, with phases between them:
//   stage 1:  z_k = sum_m' Delta_{k m'} y_m',   y_m' = (-i)^m' e^{-i m' gamma} a_m'
//   stage 2:  v_m = sum_k Delta_{k m} w_k,      w_k = e^{-i k beta} z_k,   a'_m = i^m e^{-i m alpha} v_m
// Every vector is the coefficient set of a real field (x_{-m} = (-1)^m x*_m), so with
// Delta_{j,-i} = (-1)^(l+j) Delta_{j,i} and Delta_{i,j} = (-1)^(j-i) Delta_{j,i} both stages reduce to
// sums over i >= 0 of real products:
//   S_e(j) = sum_{i: l+i+j even} Delta_{j,i} R_i,   S_o(j) = sum_{i: l+i+j odd} Delta_{j,i} I_i,
//   R_i = 2 Re x_i, I_i = 2 Im x_i (i > 0), R_0 = Re x_0, I_0 = 0,
//   stage 1: z_j = S_e + i S_o,   stage 2: v_j = (-1)^l (S_e - i S_o).
// Delta_{j,i} for fixed (l, j) follows from the three-term recurrence in the second index at
// beta = pi/2,
//   Delta_{j,i-1} = (-2 j Delta_{j,i} - sqrt((l-i)(l+i+1)) Delta_{j,i+1}) / sqrt((l+i)(l-i+1)),
// run downward from the closed form Delta_{j,l} = sqrt(C(2l, l+j)) 2^-l: from the edge inwards the
// wanted solution grows through the classically forbidden zone (i^2 + j^2 > l^2), which is the
// stable direction, and stays bounded in the oscillating zone.  Values far below the first
// significant one are carried as mantissa x 2^(F k), k < 0, and contribute nothing while k < 0.
//
// One CTA per (degree l, block of 512 outputs j): 128 threads with four outputs each walk i = l..0
// in lockstep, reading the staged inputs and recurrence coefficients of each chunk of 512 i from
// shared memory by broadcast; the sums stay in registers.  (Staging per warp instead, to spare the
// warps the per-chunk barrier, measured 7 % slower: four times the staging work, fewer warps.)  Work per stage: (l+1)^2 recurrence steps
// per degree, each a multiply and a multiply-add (normalised form, see k_rot_coef) and one
// multiply-add per coefficient set, on pairs of outputs (FP32x2 instructions in the FP32 form).
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "psht_common.cuh"
#include "psht_internal.h"

namespace psht {

namespace {

constexpr int kRotNT = 128;              // threads per CTA
constexpr int kRotNPAIR = 2;             // output pairs per thread (even)
constexpr int kRotKPT = 2 * kRotNPAIR;   // outputs j per thread
constexpr int kRotJB = kRotNT * kRotKPT; // outputs per CTA
constexpr int kRotCH = 512;              // i values staged per chunk

template <typename T>
struct RotScale;
// A value is held as d 2^(F k), k <= 0, |d| <= 2^B after each rescale test (every 8 steps); while
// k < 0 its true size is below 2^(B - F) times the growth of 8 steps (< 2^68 for lmax < 65535, one
// step grows a value by at most sqrt(2 l) + 1), so it is dropped.  FP32: B = 20, F = 120 (dropped
// below 2^-32; mantissas stay above 2^-109 after a rescale); FP64: B = 300, F = 600.
template <>
struct RotScale<float> {
  static constexpr double LOG_BIG = 20.0, LOG_STEP = 120.0;
  __device__ static float big() { return 0x1p20f; }
  __device__ static float step() { return 0x1p-120f; }
};
template <>
struct RotScale<double> {
  static constexpr double LOG_BIG = 300.0, LOG_STEP = 600.0;
  __device__ static double big() { return 0x1p300; }
  __device__ static double step() { return 0x1p-600; }
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using V = float4;
};
template <>
struct Vec4<double> {
  using V = double4_32a;
};

__host__ __device__ inline int64_t tri_off(int l) { return (int64_t)l * (l + 1) / 2; }
__host__ __device__ inline int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// Coefficients of the recurrence in the second index, per (l, i), degree-major triangle, in the
// normalised form used by the kernels.  With p_i = -2 / sqrt((l+i)(l-i+1)) and
// q_i = sqrt((l-i)(l+i+1)) / sqrt((l+i)(l-i+1)) the recurrence reads
//   Delta_{i-1} = j p_i Delta_i - q_i Delta_{i+1}.
// Writing Delta_i = s_i sigma_i u_i with sigma_l = sigma_{l-1} = 1, sigma_{i-1} = q_i sigma_{i+1}
// (so sigma lies in (0, 1]: about 0.13 at l = 4096) and s_i = (-1)^floor((l-i)/2) turns it into
//   u_{i-1} = j c.x_i u_i + u_{i+1},   c.x_i = p_i (sigma_i / sigma_{i-1}) (s_{i-1} / s_i),
// one multiply and one multiply-add per step, and the products Delta_i W_i into u_i (c.y_i W_i),
// c.y_i = s_i sigma_i, folded into the staged inputs.  One thread per degree (the sigma chain is
// sequential), FP64.
template <typename T>
__global__ void k_rot_coef(int lmax, typename Cx<T>::V* __restrict__ coef) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
    typename Cx<T>::V* cf = coef + tri_off(l);
    double sig_up = 1.0, sig = 1.0;  // sigma_{i+1}, sigma_i
    for (int i = l; i >= 1; --i) {
      const double den = 1.0 / sqrt((double)(l + i) * (double)(l - i + 1));
      const double p = -2.0 * den;
      const double q = sqrt((double)(l - i) * (double)(l + i + 1)) * den;
      const double sig_dn = (i == l) ? 1.0 : q * sig_up;  // sigma_{i-1}
      const double si = (((l - i) >> 1) & 1) ? -1.0 : 1.0, sd = (((l - i + 1) >> 1) & 1) ? -1.0 : 1.0;
      cf[i] = mk((T)(p * (sig / sig_dn) * (sd * si)), (T)(si * sig));
      sig_up = sig;
      sig = sig_dn;
    }
    const double s0 = ((l >> 1) & 1) ? -1.0 : 1.0;
    cf[0] = mk((T)0, (T)(s0 * sig));
  }
}

// log2(n!) for n = 0 .. nmax
__global__ void k_rot_logfact(int nmax, double* __restrict__ lf) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n <= nmax; n += gridDim.x * blockDim.x)
    lf[n] = lgamma((double)n + 1.0) * 1.4426950408889634;  // / ln 2
}

// phase tables: [0, L1): i^m e^{-i m alpha};  [L1, 2 L1): e^{-i k beta};  [2 L1, 3 L1): (-i)^m e^{-i m gamma}
template <typename T>
__global__ void k_rot_phases(int lmax, double alpha, double beta, double gamma, typename Cx<T>::V* __restrict__ ph) {
  const int L1 = lmax + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * L1; t += gridDim.x * blockDim.x) {
    const int which = t / L1, m = t - which * L1;
    const double ang = which == 0 ? alpha : which == 1 ? beta : gamma;
    double s, c;
    sincos(-(double)m * ang, &s, &c);
    // multiply by i^m (which 0) or (-i)^m (which 2)
    const int q = which == 0 ? (m & 3) : which == 2 ? ((4 - (m & 3)) & 3) : 0;
    double re = c, im = s;
    for (int r = 0; r < q; ++r) {
      const double t2 = re;
      re = -im;
      im = t2;
    }
    ph[t] = mk((T)re, (T)im);
  }
}

// packed pair arithmetic: two outputs per register pair (FP32x2 instructions for float)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }

// One contraction stage.  STAGE 1 reads the packed m-major input a[alm_base(i) + l] and writes
// z[tri_off(l) + j]; STAGE 2 reads z[tri_off(l) + i] and writes a'[alm_base(j) + l].
// pre[i] multiplies the input, post[j] the output (STAGE 2 only).  msc weighs the inputs i > 0
// (STAGE 1) or the outputs j > 0 (STAGE 2): the packed-gradient conventions of the plan entry points.
// Thread t owns outputs j0 + r, j0 = jfirst + 2 P t, r = 0..2P-1 (P = kRotNPAIR, even), held as P
// pairs: pair k = (r = k, r = k + P), so both members of a pair have the parity of k and read the
// same staged input.
template <typename T, int STAGE, int NSET>
__global__ void __launch_bounds__(kRotNT) k_rot_stage(int lmax, const typename Cx<T>::V* __restrict__ in0,
                                                       const typename Cx<T>::V* __restrict__ in1,
                                                       typename Cx<T>::V* __restrict__ out0,
                                                       typename Cx<T>::V* __restrict__ out1,
                                                       const typename Cx<T>::V* __restrict__ coef,
                                                       const double* __restrict__ lf,
                                                       const typename Cx<T>::V* __restrict__ pre,
                                                       const typename Cx<T>::V* __restrict__ post, T msc) {
  using V = typename Cx<T>::V;
  using V4 = typename Vec4<T>::V;
  const int l = lmax - (int)blockIdx.y;
  const int jfirst = (int)blockIdx.x * kRotJB;
  if (jfirst > l) return;
  __shared__ V4 sW[kRotCH];  // per i: (W0 set 0, W1 set 0, W0 set 1, W1 set 1), times c.y_i
  __shared__ T sC[kRotCH];   // per i: recurrence coefficient c.x_i
  const int tid = threadIdx.x;
  const int j0 = jfirst + kRotKPT * tid;

  constexpr int NP = kRotNPAIR;
  V u[NP], un[NP], mj[NP], acc[NP][2][NSET];  // [pair][parity of l+i][set]
  int ex[NP][2];                               // scale exponent of each pair member
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    T uu[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = j0 + k + NP * h;
      ex[k][h] = 0;
      uu[h] = (T)0;
      if (j <= l) {
        // log2 Delta_{j,l} = log2 sqrt(C(2l, l+j)) - l  (u_l = Delta_{j,l}: s_l = sigma_l = 1)
        double x = 0.5 * (lf[2 * l] - lf[l + j] - lf[l - j]) - (double)l;
        constexpr double low = RotScale<T>::LOG_BIG - RotScale<T>::LOG_STEP;
        if (x < low) {  // bring the mantissa into [2^low, 2^B)
          const double nres = ceil((low - x) / RotScale<T>::LOG_STEP);
          x += nres * RotScale<T>::LOG_STEP;
          ex[k][h] = -(int)nres;
        }
        uu[h] = (T)exp2(x);
      }
    }
    u[k] = mk(uu[0], uu[1]);
    un[k] = mk((T)0, (T)0);
    mj[k] = mk((T)(j0 + k), (T)(j0 + k + NP));
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int s = 0; s < NSET; ++s) acc[k][p][s] = mk((T)0, (T)0);
  }
  bool fast = false;  // every output of this warp is at scale 0: no gate, no rescale test

  auto rescale = [&]() {
    bool all0 = true;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (fabs(u[k].x) > RotScale<T>::big()) {
        u[k].x *= RotScale<T>::step();
        un[k].x *= RotScale<T>::step();
        ex[k][0] += 1;
      }
      if (fabs(u[k].y) > RotScale<T>::big()) {
        u[k].y *= RotScale<T>::step();
        un[k].y *= RotScale<T>::step();
        ex[k][1] += 1;
      }
      all0 = all0 && ex[k][0] == 0 && ex[k][1] == 0;
    }
    return all0;
  };

  for (int ihi = l; ihi >= 0; ihi -= kRotCH) {
    const int ilo = max(0, ihi - kRotCH + 1);
    // stage inputs and coefficients of i in [ilo, ihi]
    for (int i = ilo + tid; i <= ihi; i += kRotNT) {
      V x0, x1 = mk((T)0, (T)0);
      if (STAGE == 1) {
        const int64_t k = alm_base(lmax, i) + l;
        x0 = in0[k];
        if (NSET == 2) x1 = in1[k];
      } else {
        const int64_t k = tri_off(l) + i;
        x0 = in0[k];
        if (NSET == 2) x1 = in1[k];
      }
      const V ph = pre[i];
      const V c = coef[tri_off(l) + i];
      x0 = cmul(x0, ph);
      x1 = cmul(x1, ph);
      const T two = (i == 0 ? (T)1 : (STAGE == 1 ? (T)2 * msc : (T)2)) * c.y;
      const T R0 = two * x0.x, I0 = i == 0 ? (T)0 : two * x0.y;
      const T R1 = two * x1.x, I1 = i == 0 ? (T)0 : two * x1.y;
      const bool odd = ((l + i) & 1) != 0;
      V4 w;
      w.x = odd ? I0 : R0;
      w.y = odd ? R0 : I0;
      w.z = odd ? I1 : R1;
      w.w = odd ? R1 : I1;
      sW[i - ilo] = w;
      sC[i - ilo] = c.x;
    }
    __syncthreads();

    // one step at index i, parity P = (l + i) & 1 (the chunk starts at even parity: l + ihi is even
    // for ihi = l - 512 c)
    auto step = [&](int i, int P, bool gated) {
      const V4 w = sW[i - ilo];
      const T cx = sC[i - ilo];
      const V cx2 = mk(cx, cx);
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        V dv = u[k];
        if (gated) {
          if (ex[k][0] != 0) dv.x = (T)0;
          if (ex[k][1] != 0) dv.y = (T)0;
        }
        const T wa = (k & 1) ? w.y : w.x;
        acc[k][P][0] = fma2(dv, mk(wa, wa), acc[k][P][0]);
        if (NSET == 2) {
          const T wb = (k & 1) ? w.w : w.z;
          acc[k][P][NSET - 1] = fma2(dv, mk(wb, wb), acc[k][P][NSET - 1]);
        }
        const V nu = fma2(mul2(mj[k], cx2), u[k], un[k]);
        un[k] = u[k];
        u[k] = nu;
      }
    };
    int i = ihi;
    // gated steps in blocks of 8 with a rescale test after each block, until the warp is at scale 0
    while (!fast && i >= ilo + 7) {
#pragma unroll
      for (int u8 = 0; u8 < 8; u8 += 2) {
        step(i - u8, 0, true);
        step(i - u8 - 1, 1, true);
      }
      i -= 8;
      fast = __all_sync(0xffffffffu, rescale());
    }
    if (fast) {
      for (; i >= ilo + 1; i -= 2) {
        step(i, 0, false);
        step(i - 1, 1, false);
      }
    } else {
      // fewer than 8 steps left in this chunk: gated, then a rescale test
      for (; i >= ilo + 1; i -= 2) {
        step(i, 0, true);
        step(i - 1, 1, true);
      }
      rescale();
    }
    if (i == ilo) step(i, 0, !fast);
    __syncthreads();
  }

  // outputs: for even j, S_e = acc[.][0], S_o = acc[.][1]; for odd j the other way round
#pragma unroll
  for (int k = 0; k < NP; ++k) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = j0 + k + NP * h;
      if (j > l) continue;
#pragma unroll
      for (int s = 0; s < NSET; ++s) {
        const V ae = (k & 1) ? acc[k][1][s] : acc[k][0][s];
        const V ao = (k & 1) ? acc[k][0][s] : acc[k][1][s];
        const T Se = h ? ae.y : ae.x, So = h ? ao.y : ao.x;
        V* out = s == 0 ? out0 : out1;
        if (STAGE == 1) {
          out[tri_off(l) + j] = mk(Se, So);
        } else {
          const T sg = (l & 1) ? (T)-1 : (T)1;
          V v = cmul(mk(sg * Se, -sg * So), post[j]);
          if (j == 0) v.y = (T)0;
          else v = cscale(v, msc);
          out[alm_base(lmax, j) + l] = v;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// points: n = R p, (theta', phi'), and psi = angle from e_theta(p) towards e_phi(p) of R^-1 e_theta'(n)
struct Mat3 {
  double a[9];
};

__global__ void k_rot_points(Mat3 R, const double* __restrict__ theta, const double* __restrict__ phi, int64_t n,
                             double* __restrict__ theta2, double* __restrict__ phi2, double* __restrict__ psi) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double st, ct, sp, cp;
    sincos(theta[p], &st, &ct);
    sincos(phi[p], &sp, &cp);
    const double v0 = st * cp, v1 = st * sp, v2 = ct;
    const double n0 = R.a[0] * v0 + R.a[1] * v1 + R.a[2] * v2;
    const double n1 = R.a[3] * v0 + R.a[4] * v1 + R.a[5] * v2;
    const double n2 = R.a[6] * v0 + R.a[7] * v1 + R.a[8] * v2;
    const double rho = hypot(n0, n1);
    const double th2 = atan2(rho, n2);
    double ph2 = atan2(n1, n0);
    if (ph2 < 0.0) ph2 += 2.0 * M_PI;
    if (ph2 >= 2.0 * M_PI) ph2 -= 2.0 * M_PI;
    theta2[p] = th2;
    phi2[p] = ph2;
    if (psi) {
      // e_theta' at n in the rotated frame, then R^T of it
      double s2, c2, sq, cq;
      sincos(th2, &s2, &c2);
      sincos(ph2, &sq, &cq);
      const double e0 = c2 * cq, e1 = c2 * sq, e2 = -s2;
      const double b0 = R.a[0] * e0 + R.a[3] * e1 + R.a[6] * e2;
      const double b1 = R.a[1] * e0 + R.a[4] * e1 + R.a[7] * e2;
      const double b2 = R.a[2] * e0 + R.a[5] * e1 + R.a[8] * e2;
      const double dt = b0 * ct * cp + b1 * ct * sp - b2 * st;  // . e_theta(p)
      const double dp = -b0 * sp + b1 * cp;                     // . e_phi(p)
      psi[p] = atan2(dp, dt);
    }
  }
}

// e^{i s psi_p} per point, in the plan's precision
template <typename T>
__global__ void k_spin_phase(const double* __restrict__ psi, int s, int64_t n, typename Cx<T>::V* __restrict__ ph) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double sn, cs;
    sincos((double)s * psi[p], &sn, &cs);
    ph[p] = mk((T)cs, (T)sn);
  }
}

// out_p = in_p ph_p (CONJ: in_p conj(ph_p)); out may alias in
template <typename T, bool CONJ>
__global__ void k_mul_phase(const typename Cx<T>::V* in, const typename Cx<T>::V* __restrict__ ph, int64_t n,
                            typename Cx<T>::V* out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    out[p] = CONJ ? cmulc(in[p], ph[p]) : cmul(in[p], ph[p]);
}

// ---------------------------------------------------------------------------------------------
// linear minimisation over the points: argmin_p <p, x>, FP32 dot products for the search; the
// winner is returned with its FP64 unit vector
struct LmoOut {
  double v[3];
  double dot;
  int64_t idx;
};

constexpr int kLmoThreads = 256;

__global__ void k_lmo_partial(const double* __restrict__ theta, const double* __restrict__ phi, int64_t n, float x0,
                              float x1, float x2, float* __restrict__ pval, int64_t* __restrict__ pidx) {
  float best = INFINITY;
  int64_t bi = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float st, ct, sp, cp;
    sincosf((float)theta[p], &st, &ct);
    sincosf((float)phi[p], &sp, &cp);
    const float v = x0 * st * cp + x1 * st * sp + x2 * ct;
    if (v < best) {
      best = v;
      bi = p;
    }
  }
  __shared__ float sv[kLmoThreads];
  __shared__ int64_t si[kLmoThreads];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int h = kLmoThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h && sv[threadIdx.x + h] < sv[threadIdx.x]) {
      sv[threadIdx.x] = sv[threadIdx.x + h];
      si[threadIdx.x] = si[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pval[blockIdx.x] = sv[0];
    pidx[blockIdx.x] = si[0];
  }
}

__global__ void k_lmo_final(const double* __restrict__ theta, const double* __restrict__ phi, int nb,
                            const float* __restrict__ pval, const int64_t* __restrict__ pidx, double x0, double x1,
                            double x2, LmoOut* __restrict__ out) {
  __shared__ float sv[kLmoThreads];
  __shared__ int64_t si[kLmoThreads];
  float best = INFINITY;
  int64_t bi = 0;
  for (int b = threadIdx.x; b < nb; b += kLmoThreads)
    if (pval[b] < best) {
      best = pval[b];
      bi = pidx[b];
    }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int h = kLmoThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h && sv[threadIdx.x + h] < sv[threadIdx.x]) {
      sv[threadIdx.x] = sv[threadIdx.x + h];
      si[threadIdx.x] = si[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t p = si[0];
    double st, ct, sp, cp;
    sincos(theta[p], &st, &ct);
    sincos(phi[p], &sp, &cp);
    out->v[0] = st * cp;
    out->v[1] = st * sp;
    out->v[2] = ct;
    out->dot = x0 * out->v[0] + x1 * out->v[1] + x2 * out->v[2];
    out->idx = p;
  }
}

struct V3 {
  double x, y, z;
};
inline double dot3(const V3& a, const V3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// affine minimiser of |sum mu_i s_i|^2 subject to sum mu_i = 1 (k <= 4 points), by the bordered
// normal equations with partial pivoting; false if singular
bool affine_min(const std::vector<V3>& S, std::vector<double>& mu) {
  const int k = (int)S.size();
  double A[5][6];
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j < k; ++j) A[i][j] = dot3(S[i], S[j]);
    A[i][k] = 1.0;
    A[i][k + 1] = 0.0;
  }
  for (int j = 0; j < k; ++j) A[k][j] = 1.0;
  A[k][k] = 0.0;
  A[k][k + 1] = 1.0;
  const int n = k + 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (fabs(A[piv][c]) < 1e-300) return false;
    if (piv != c)
      for (int j = 0; j <= n; ++j) std::swap(A[c][j], A[piv][j]);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r][c] / A[c][c];
      for (int j = c; j <= n; ++j) A[r][j] -= f * A[c][j];
    }
  }
  mu.resize(k);
  for (int i = 0; i < k; ++i) mu[i] = A[i][n] / A[i][i];
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
struct Rotator {
  int lmax = 0, prec = 64;
  int64_t nalm = 0;
  void* d_coef = nullptr;  // T2 [tri_off(lmax+1)]
  double* d_lf = nullptr;  // [2 lmax + 2]
  void* d_ph = nullptr;    // T2 [3 (lmax+1)]
  void* d_z = nullptr;     // T2 [2][nalm]
  size_t bytes = 0;
};

size_t rotator_bytes(int lmax, int prec) {
  const int64_t n = tri_off(lmax + 1);
  const size_t cb = prec == 64 ? 16 : 8;
  return (size_t)n * cb * 3 + (size_t)(2 * lmax + 2) * 8 + (size_t)3 * (lmax + 1) * cb;
}

Rotator* rotator_create(int lmax, int prec, cudaStream_t st) {
  PSHT_REQUIRE(lmax >= 0 && lmax <= 65534, PSHT_EINVAL, "rotation: lmax must lie in [0, 65534]");
  PSHT_REQUIRE(prec == 32 || prec == 64, PSHT_EINVAL, "rotation: precision must be PSHT_FP32 or PSHT_FP64");
  Rotator* r = new Rotator;
  r->lmax = lmax;
  r->prec = prec;
  r->nalm = tri_off(lmax + 1);
  const size_t cb = prec == 64 ? 16 : 8;
  auto fail = [&](cudaError_t e) {
    rotator_destroy(r);
    throw Error{e == cudaErrorMemoryAllocation ? PSHT_ENOMEM : PSHT_ECUDA,
                std::string("rotation: ") + cudaGetErrorString(e)};
  };
  cudaError_t e;
  if ((e = cudaMalloc(&r->d_coef, (size_t)r->nalm * cb)) != cudaSuccess) fail(e);
  if ((e = cudaMalloc((void**)&r->d_lf, (size_t)(2 * lmax + 2) * 8)) != cudaSuccess) fail(e);
  if ((e = cudaMalloc(&r->d_ph, (size_t)3 * (lmax + 1) * cb)) != cudaSuccess) fail(e);
  if ((e = cudaMalloc(&r->d_z, (size_t)2 * r->nalm * cb)) != cudaSuccess) fail(e);
  r->bytes = rotator_bytes(lmax, prec);
  const int nb = (lmax + 64) / 64;
  if (prec == 64) k_rot_coef<double><<<nb, 64, 0, st>>>(lmax, (double2*)r->d_coef);
  else k_rot_coef<float><<<nb, 64, 0, st>>>(lmax, (float2*)r->d_coef);
  k_rot_logfact<<<(2 * lmax + 2 + 255) / 256, 256, 0, st>>>(2 * lmax + 1, r->d_lf);
  if ((e = cudaGetLastError()) != cudaSuccess) fail(e);
  return r;
}

void rotator_destroy(Rotator* r) {
  if (!r) return;
  cudaFree(r->d_coef);
  cudaFree(r->d_lf);
  cudaFree(r->d_ph);
  cudaFree(r->d_z);
  delete r;
}

int rotator_lmax(const Rotator* r) { return r->lmax; }
int rotator_prec(const Rotator* r) { return r->prec; }

template <typename T>
static void apply_t(Rotator& r, double alpha, double beta, double gamma, const void* g, const void* c, void* go,
                    void* co, cudaStream_t st, double in_msc, double out_msc) {
  using V = typename Cx<T>::V;
  const int lmax = r.lmax, L1 = lmax + 1;
  V* ph = (V*)r.d_ph;
  k_rot_phases<T><<<(3 * L1 + 255) / 256, 256, 0, st>>>(lmax, alpha, beta, gamma, ph);
  const dim3 grid((unsigned)((lmax + kRotJB) / kRotJB), (unsigned)L1);
  V* z0 = (V*)r.d_z;
  V* z1 = z0 + r.nalm;
  const V* cf = (const V*)r.d_coef;
  if (c) {
    k_rot_stage<T, 1, 2><<<grid, kRotNT, 0, st>>>(lmax, (const V*)g, (const V*)c, z0, z1, cf, r.d_lf, ph + 2 * L1,
                                                  nullptr, (T)in_msc);
    k_rot_stage<T, 2, 2><<<grid, kRotNT, 0, st>>>(lmax, z0, z1, (V*)go, (V*)co, cf, r.d_lf, ph + L1, ph,
                                                  (T)out_msc);
  } else {
    k_rot_stage<T, 1, 1><<<grid, kRotNT, 0, st>>>(lmax, (const V*)g, nullptr, z0, nullptr, cf, r.d_lf, ph + 2 * L1,
                                                  nullptr, (T)in_msc);
    k_rot_stage<T, 2, 1><<<grid, kRotNT, 0, st>>>(lmax, z0, nullptr, (V*)go, nullptr, cf, r.d_lf, ph + L1, ph,
                                                  (T)out_msc);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

void rotator_apply(Rotator& r, double alpha, double beta, double gamma, const void* g, const void* c, void* go,
                   void* co, cudaStream_t st, double in_msc, double out_msc) {
  PSHT_REQUIRE(g && go, PSHT_EINVAL, "rotation: g and g_out must not be NULL");
  PSHT_REQUIRE((c == nullptr) == (co == nullptr), PSHT_EINVAL, "rotation: c and c_out must both be set or both NULL");
  PSHT_REQUIRE(std::isfinite(alpha) && std::isfinite(beta) && std::isfinite(gamma), PSHT_EINVAL,
               "rotation: Euler angles must be finite");
  if (r.prec == 64) apply_t<double>(r, alpha, beta, gamma, g, c, go, co, st, in_msc, out_msc);
  else apply_t<float>(r, alpha, beta, gamma, g, c, go, co, st, in_msc, out_msc);
}

static Mat3 rotation_matrix(double alpha, double beta, double gamma) {
  const double ca = cos(alpha), sa = sin(alpha), cb = cos(beta), sb = sin(beta), cg = cos(gamma), sg = sin(gamma);
  // R_z(alpha) R_y(beta) R_z(gamma)
  Mat3 R;
  R.a[0] = ca * cb * cg - sa * sg;
  R.a[1] = -ca * cb * sg - sa * cg;
  R.a[2] = ca * sb;
  R.a[3] = sa * cb * cg + ca * sg;
  R.a[4] = -sa * cb * sg + ca * cg;
  R.a[5] = sa * sb;
  R.a[6] = -sb * cg;
  R.a[7] = sb * sg;
  R.a[8] = cb;
  return R;
}

void rotate_points_device(double alpha, double beta, double gamma, const double* theta, const double* phi,
                          int64_t n, double* theta2, double* phi2, double* psi, cudaStream_t st) {
  PSHT_REQUIRE(n >= 0, PSHT_EINVAL, "rotation: npts must be >= 0");
  PSHT_REQUIRE(n == 0 || (theta && phi && theta2 && phi2), PSHT_EINVAL, "rotation: point arrays must not be NULL");
  PSHT_REQUIRE(std::isfinite(alpha) && std::isfinite(beta) && std::isfinite(gamma), PSHT_EINVAL,
               "rotation: Euler angles must be finite");
  if (n == 0) return;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_rot_points<<<nb, 256, 0, st>>>(rotation_matrix(alpha, beta, gamma), theta, phi, n, theta2, phi2, psi);
  PSHT_CUDA_TRY(cudaGetLastError());
}

void spin_phase_device(int prec, const double* psi, int s, int64_t n, void* ph, cudaStream_t st) {
  if (n <= 0) return;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  if (prec == 64) k_spin_phase<double><<<nb, 256, 0, st>>>(psi, s, n, (double2*)ph);
  else k_spin_phase<float><<<nb, 256, 0, st>>>(psi, s, n, (float2*)ph);
  PSHT_CUDA_TRY(cudaGetLastError());
}

void mul_phase_device(int prec, const void* in, const void* ph, int64_t n, bool conj, void* out, cudaStream_t st) {
  if (n <= 0) return;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  if (prec == 64) {
    if (conj) k_mul_phase<double, true><<<nb, 256, 0, st>>>((const double2*)in, (const double2*)ph, n, (double2*)out);
    else k_mul_phase<double, false><<<nb, 256, 0, st>>>((const double2*)in, (const double2*)ph, n, (double2*)out);
  } else {
    if (conj) k_mul_phase<float, true><<<nb, 256, 0, st>>>((const float2*)in, (const float2*)ph, n, (float2*)out);
    else k_mul_phase<float, false><<<nb, 256, 0, st>>>((const float2*)in, (const float2*)ph, n, (float2*)out);
  }
  PSHT_CUDA_TRY(cudaGetLastError());
}

// Wolfe's minimum-norm-point iteration over the points' convex hull; the linear minimisations run
// on the device.  Returns the Euler angles (0, theta_c, pi - phi_c) of the rotation taking the cap
// centre c to the north pole, and the cap radius.
void patch_rotation_device(const double* theta, const double* phi, int64_t n, double euler[3], double* theta_star,
                           cudaStream_t st) {
  PSHT_REQUIRE(n > 0 && theta && phi && euler, PSHT_EINVAL, "patch rotation: need at least one point");
  const int nb = (int)std::min<int64_t>((n + kLmoThreads - 1) / kLmoThreads, 152 * 8);
  float* d_val = nullptr;
  int64_t* d_idx = nullptr;
  LmoOut* d_out = nullptr;
  auto cleanup = [&] {
    cudaFree(d_val);
    cudaFree(d_idx);
    cudaFree(d_out);
  };
  try {
    PSHT_CUDA_TRY(cudaMalloc((void**)&d_val, (size_t)nb * sizeof(float)));
    PSHT_CUDA_TRY(cudaMalloc((void**)&d_idx, (size_t)nb * sizeof(int64_t)));
    PSHT_CUDA_TRY(cudaMalloc((void**)&d_out, sizeof(LmoOut)));
    auto lmo = [&](const V3& x) {
      k_lmo_partial<<<nb, kLmoThreads, 0, st>>>(theta, phi, n, (float)x.x, (float)x.y, (float)x.z, d_val, d_idx);
      k_lmo_final<<<1, kLmoThreads, 0, st>>>(theta, phi, nb, d_val, d_idx, x.x, x.y, x.z, d_out);
      PSHT_CUDA_TRY(cudaGetLastError());
      LmoOut h;
      PSHT_CUDA_TRY(cudaMemcpyAsync(&h, d_out, sizeof(LmoOut), cudaMemcpyDeviceToHost, st));
      PSHT_CUDA_TRY(cudaStreamSynchronize(st));
      return h;
    };
    // start from the point farthest along -z (any point of the hull would do)
    LmoOut h0 = lmo(V3{0.0, 0.0, 1.0});
    std::vector<V3> S{V3{h0.v[0], h0.v[1], h0.v[2]}};
    std::vector<int64_t> Sidx{h0.idx};
    std::vector<double> lam{1.0}, mu;
    V3 x = S[0];
    for (int major = 0; major < 200; ++major) {
      const LmoOut h = lmo(x);
      const double xx = dot3(x, x);
      if (xx - h.dot <= 1e-12 * std::max(xx, 1e-300)) break;
      if (std::find(Sidx.begin(), Sidx.end(), h.idx) != Sidx.end()) break;
      if (S.size() == 4) break;  // cannot happen for points in an open hemisphere
      S.push_back(V3{h.v[0], h.v[1], h.v[2]});
      Sidx.push_back(h.idx);
      lam.push_back(0.0);
      for (int minor = 0; minor < 16; ++minor) {
        if (!affine_min(S, mu)) break;
        bool inside = true;
        for (double m : mu) inside = inside && m > 1e-14;
        if (inside) {
          lam = mu;
          break;
        }
        double th = 1.0;
        for (size_t i = 0; i < S.size(); ++i)
          if (mu[i] <= 1e-14) th = std::min(th, lam[i] / std::max(lam[i] - mu[i], 1e-300));
        for (size_t i = 0; i < S.size(); ++i) lam[i] = (1.0 - th) * lam[i] + th * mu[i];
        for (size_t i = S.size(); i-- > 0;)
          if (lam[i] <= 1e-14) {
            S.erase(S.begin() + i);
            Sidx.erase(Sidx.begin() + i);
            lam.erase(lam.begin() + i);
          }
        double tot = 0.0;
        for (double v : lam) tot += v;
        for (double& v : lam) v /= tot;
      }
      x = V3{0.0, 0.0, 0.0};
      for (size_t i = 0; i < S.size(); ++i) {
        x.x += lam[i] * S[i].x;
        x.y += lam[i] * S[i].y;
        x.z += lam[i] * S[i].z;
      }
    }
    const double nx = sqrt(dot3(x, x));
    PSHT_REQUIRE(nx > 1e-9, PSHT_EINVAL, "patch rotation: the points do not lie in an open hemisphere");
    const V3 cdir{x.x / nx, x.y / nx, x.z / nx};
    const LmoOut h = lmo(cdir);
    const double tc = atan2(hypot(cdir.x, cdir.y), cdir.z);
    double pc = atan2(cdir.y, cdir.x);
    euler[0] = 0.0;
    euler[1] = tc;
    euler[2] = M_PI - pc;
    if (theta_star) *theta_star = acos(std::min(1.0, std::max(-1.0, h.dot)));
    cleanup();
  } catch (...) {
    cleanup();
    throw;
  }
}

}  // namespace psht
