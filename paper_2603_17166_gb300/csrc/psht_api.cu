// Planner (host) and the C-ABI entry points of include/psht.h.
//
// The planner follows Sec. II of Carron & Reinecke (steps 1-4) and the parameter choice of
// Sec. II.C-D, plus the numerical choices the paper leaves open (ring count rounding, polar
// optimisation cutoff, NUFFT grid), which the FP64 CPU oracle states identically.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <initializer_list>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "psht_internal.h"

namespace psht {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

void allow_dynamic_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> granted;  // (kernel, device) -> bytes allowed
  int dev = 0;
  PSHT_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(fn, dev);
  auto it = granted.find(key);
  if (it == granted.end()) {
    cudaFuncAttributes fa;
    PSHT_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
    int optin = 0;
    PSHT_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int most = optin - (int)fa.sharedSizeBytes;
    PSHT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
    it = granted.emplace(key, (size_t)std::max(most, 0)).first;
  }
  PSHT_REQUIRE(bytes <= it->second, PSHT_ENOTSUP,
               "a kernel needs " + std::to_string(bytes) + " B of shared memory, above the device's " +
                   std::to_string(it->second));
}

namespace {

// ---------------------------------------------------------------------------------------------
// small numerical helpers
int fft_friendly(int n) {
  n = std::max(n, 1);
  for (;; ++n) {
    int k = n;
    for (int p : {2, 3, 5, 7})
      while (k % p == 0) k /= p;
    if (k == 1) return n;
  }
}

FftDev radix_schedule(int n) {
  FftDev f{};
  f.n = n;
  int k = n, st = 0;
  auto push = [&](int r) { f.rad[st++] = r; k /= r; };
  while (k % 8 == 0) push(8);
  while (k % 4 == 0) push(4);
  while (k % 2 == 0) push(2);
  for (int p : {3, 5, 7})
    while (k % p == 0) push(p);
  PSHT_REQUIRE(k == 1 && st <= 32, PSHT_ENOTSUP, "FFT length has a prime factor above 7");
  f.nst = st;
  return f;
}

// DIF output position of frequency k: sum_i q_i s_i, q_i = (k / (R_1..R_{i-1})) mod R_i, s_i = N/(R_1..R_i)
std::vector<int> fft_perm(const FftDev& f) {
  std::vector<int> pos(f.n);
  for (int k0 = 0; k0 < f.n; ++k0) {
    int k = k0, p = 0, s = f.n;
    for (int i = 0; i < f.nst; ++i) {
      s /= f.rad[i];
      p += (k % f.rad[i]) * s;
      k /= f.rad[i];
    }
    pos[k0] = p;
  }
  return pos;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Quad {
  std::vector<double> x, w;
  Quad() { gauss_legendre(256, x, w); }
  template <class F>
  double integrate(F f, double a, double b) const {
    const double xm = 0.5 * (a + b), xr = 0.5 * (b - a);
    double s = 0;
    for (size_t i = 0; i < x.size(); ++i) s += w[i] * f(xm + xr * x[i]);
    return xr * s;
  }
};

// modified Bessel function I0(x) e^{-x} for 0 <= x <= ~50 by its power series sum (x^2/4)^k/(k!)^2
double bessel_i0_scaled(double x) {
  const double q = 0.25 * x * x;
  double term = exp(-x), sum = term;
  for (int k = 1; k < 200; ++k) {
    term *= q / ((double)k * k);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

// window w(Theta) = B(pi - dTheta/2 - |Theta|), B the CDF of the unit-area bell of support dTheta
// (Sec. II.D): the ES bell exp[c (sqrt(1 - v^2) - 1)] or the Kaiser-Bessel bell I0(c sqrt(1 - v^2)),
// v = 2u/dTheta, c = alpha pi = |ln eps|; u = (dTheta/2) sin(tau) makes the integrand smooth.
double window_value(double Theta, double dTheta, double cexp, int kind, const Quad& q) {
  const double x = M_PI - 0.5 * dTheta - fabs(Theta);
  const double z = 2.0 * x / dTheta;
  if (z <= -1.0) return 0.0;
  if (z >= 1.0) return 1.0;
  auto dens = [&](double tau) {
    const double c = cos(tau);
    return (kind == PSHT_WINDOW_KB ? bessel_i0_scaled(cexp * c) * exp(cexp * (c - 1.0)) : exp(cexp * (c - 1.0))) * c;
  };
  return q.integrate(dens, -0.5 * M_PI, asin(z)) / q.integrate(dens, -0.5 * M_PI, 0.5 * M_PI);
}

// continuous FT of psi(x/a), a = W pi/nfine, at integer frequency k
double es_ft(double k, int W, double beta, int nfine, const Quad& q) {
  const double a = W * M_PI / nfine;
  auto f = [&](double tau) { return exp(beta * (cos(tau) - 1.0)) * cos(k * a * sin(tau)) * cos(tau); };
  return a * q.integrate(f, -0.5 * M_PI, 0.5 * M_PI);
}

int es_width(double eps) { return std::min(16, (int)ceil(-log10(eps) - 1e-9) + 1); }

// polar-optimisation cutoff (Sec. II.A): turning point x = (lmax + 1/2) sin(beta) plus the
// Airy-type tail kept down to 1e-3 eps
int mcut(int lmax, int s, double eps, double beta) {
  const double z = pow(1.5 * log(1.0 / (1e-3 * eps)), 2.0 / 3.0);
  const double x = (lmax + 0.5) * fabs(sin(beta));
  const double v = ceil(x + s + 1.25 * z * pow(x / 2.0, 1.0 / 3.0) + 8.0);
  return (int)std::min<double>(lmax, v);
}

template <typename T>
void* upload(Plan& p, const std::vector<T>& h, cudaStream_t st) {
  void* d = nullptr;
  const size_t b = std::max<size_t>(1, h.size()) * sizeof(T);
  PSHT_CUDA_TRY(cudaMalloc(&d, b));
  p.allocs.push_back(d);
  p.bytes += b;
  if (!h.empty()) PSHT_CUDA_TRY(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return d;
}

void* dalloc(Plan& p, size_t b) {
  void* d = nullptr;
  b = std::max<size_t>(b, 16);
  cudaError_t e = cudaMalloc(&d, b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[160];
    snprintf(msg, sizeof(msg), "device allocation of %zu bytes failed (plan holds %zu)", b, p.bytes);
    throw Error{PSHT_ENOMEM, msg};
  }
  p.allocs.push_back(d);
  p.bytes += b;
  return d;
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

// ---------------------------------------------------------------------------------------------
// P1-P2 and the grid: everything that depends on (spin, lmax, eps, precision, theta*, pole)


// (ring, m, l) steps of the recursion on one ring with cutoff M: sum_{m=0}^{M} (lmax + 1 - max(m, s))
int64_t ring_cost(int lmax, int s, int M) {
  const int64_t n = (int64_t)(M + 1) * (lmax + 1);
  const int64_t sm = M < s ? (int64_t)(M + 1) * s : (int64_t)s * s + ((int64_t)M * (M + 1) - (int64_t)(s - 1) * s) / 2;
  return n - sm;
}

// The apodisation length minimising the recursion's step count with polar optimisation: for
// eps_apo = e the window adds Delta l pi / (e theta*) modes, Lmax(e) = kappa (lmax theta*/pi)(1 + e)
// (1 + e0^2/e), minimal at the paper's e0 (eq. Lmax2); candidates e = e0 (20 + k)/40, k = 0..80.
// False if every candidate needs the full sky.
bool cost_optimal_apo(const Plan& p, double e0, double& e_best, int& Lmax_best) {
  bool found = false;
  int64_t best = 0;
  for (int k = 0; k <= 80; ++k) {
    const double e = e0 * ((20 + k) / 40.0);
    const double tmax = p.theta_star * (1.0 + e);
    const int Lmax = (int)ceil(p.kappa * p.lmax * p.theta_star / M_PI * (1.0 + e) * (1.0 + e0 * e0 / e));
    if (tmax >= M_PI || Lmax >= p.lmax) continue;
    const int L = fft_friendly(Lmax + 1);
    int64_t cost = 0;
    for (int j = 0; j < L; ++j) {
      const double Th = j * (M_PI / L);
      cost += ring_cost(p.lmax, p.spin, mcut(p.lmax, p.spin, p.eps, Th * (tmax / M_PI)));
    }
    if (!found || cost < best) {
      found = true;
      best = cost;
      e_best = e;
      Lmax_best = Lmax;
    }
  }
  return found;
}

void layout(Plan& p, double theta_star) {
  const double lneps = fabs(log(p.eps));
  p.theta_star = std::max(theta_star, 1e-9);
  bool full = p.lmax < 1 || p.force_full;
  if (!full) {
    p.eps_apo = sqrt(2.0 * lneps / (p.theta_star * p.lmax));
    p.theta_max = p.theta_star * (1.0 + p.eps_apo);
    p.Lmax = (int)ceil(p.kappa * p.lmax * p.theta_star / M_PI * (1.0 + p.eps_apo) * (1.0 + p.eps_apo));
    if (p.theta_max >= M_PI || p.Lmax >= p.lmax) full = true;
    if (p.apo_cost) {
      double e = 0.0;
      int Lm = 0;
      full = !cost_optimal_apo(p, p.eps_apo, e, Lm);
      if (!full) {
        p.eps_apo = e;
        p.theta_max = p.theta_star * (1.0 + e);
        p.Lmax = Lm;
      }
    }
  }
  p.full = full ? 1 : 0;
  if (full) {
    p.eps_apo = 0.0;
    p.theta_max = M_PI;
    p.Lmax = p.lmax;
    p.dTheta = 0.0;
  } else {
    p.dTheta = M_PI * p.eps_apo / (1.0 + p.eps_apo);
  }
  p.alpha = lneps / M_PI;
  p.omx_tb = (p.prec == 64 && p.eps >= kThreeTermMinEps) ? 1.0 - cos(kThreeTermDeg * M_PI / 180.0) : 3.0;
  p.L = fft_friendly(p.Lmax + 1);
  p.nring = full ? p.L + 1 : p.L;
  p.theta_j.resize(p.nring);
  p.beta_j.resize(p.nring);
  p.w_j.resize(p.nring);
  p.Mj.resize(p.nring);
  static const Quad quad;
  for (int j = 0; j < p.nring; ++j) {
    const double Th = j * (M_PI / p.L);
    p.beta_j[j] = Th * (p.theta_max / M_PI);
    p.theta_j[j] = p.pole > 0 ? p.beta_j[j] : M_PI - p.beta_j[j];
    p.w_j[j] = full ? 1.0 : window_value(Th, p.dTheta, lneps, p.window, quad);
    p.Mj[j] = mcut(p.lmax, p.spin, p.eps, p.beta_j[j]);
  }
  p.M = *std::max_element(p.Mj.begin(), p.Mj.end());
  p.W = es_width(p.eps);
  p.beta_es = 2.30 * p.W;
  p.nTheta = 4 * p.L;
  p.nphi = 2 * fft_friendly(2 * p.M + 1);
  const double t_max = p.theta_star * p.nTheta / (2.0 * p.theta_max);
  p.r_lo = (int)ceil(-0.5 * p.W);
  const int r_hi = (int)ceil(t_max - 0.5 * p.W) + p.W;
  p.nrows = r_hi - p.r_lo + 1;
  p.ncols = 2 * p.M + 1;
  p.Lpad = (p.nring + 31) / 32 * 32;
  p.padq = 8;
  p.gstride = (p.nphi + 2 * p.padq + 7) / 8 * 8;
  // point tiles of TR x TQ base cells: FP32 32 x 16 (its spreading kernel gives each of a warp's
  // lanes one base row), FP64 16 x 32
  p.TR = p.prec == 32 ? 32 : 16;
  p.TQ = p.prec == 32 ? 16 : 32;
  p.ntr = (p.nrows - 1) / p.TR + 1;
  p.ntq = (p.nphi + p.padq) / p.TQ + 1;
  p.nalm = (int64_t)(p.lmax + 1) * (p.lmax + 2) / 2;
  p.tstride = p.nalm + 64;  // one chunk of zero records after the last order
  // launch shapes of the recursion
  // rings per lane of the one-warp synthesis: FP64 1, FP32 kSynRpt32 (one packed pair)
  p.syn_rpt = (p.prec == 64) ? 1 : kSynRpt32;
  p.syn_threads = 32;  // one warp per synthesis item (k_rec_syn_w)
  // adjoint.  FP32: one warp per item of 32 adj_rpt rings (k_rec_adj_w), the items of an order
  // meeting in a float4-per-coefficient accumulator.  FP64: one CTA per m and chunk of
  // adj_rpt * adj_threads rings (k_rec_adj), (rings per thread, threads) from the instantiated
  // shapes with the fewest idle ring slots.
  p.adj_rpt = p.nring <= 256 ? 2 : (p.nring <= 512 ? 4 : 8);
  p.adj_threads = 128;
  if (p.prec == 32) {
    p.adj_threads = 32;
    p.adj_rpt = 4;  // two packed pairs per lane (8 rings per lane measured slower: 128 registers)
  }
  // FFTs longer than one CTA's shared memory run on global buffers (psht_fft.cu)
  constexpr int kMaxLen = 1 << 22;
  PSHT_REQUIRE(p.nTheta <= kMaxLen && p.nphi <= kMaxLen, PSHT_ENOTSUP,
               "FFT length above " + std::to_string(kMaxLen) + " (Theta " + std::to_string(p.nTheta) + ", phi " +
                   std::to_string(p.nphi) + ")");
}

size_t planned_bytes(const Plan& p) {
  const size_t cb = p.prec == 64 ? 16 : 8, rb = p.prec == 64 ? 8 : 4;
  size_t b = 0;
  b += (size_t)rec_table_record_bytes(p.prec) * p.tstride;            // recursion table
  b += (size_t)p.ncols * p.Lpad * cb;                          // ring coefficients
  b += (size_t)p.nrows * p.ncols * cb;                         // Theta-stage rows
  b += (size_t)p.nrows * p.gstride * cb;                       // grid
  b += (size_t)p.npts * 8;                                     // index + cell
  b += p.prec == 64 ? (size_t)p.npts * 2 * p.W * 8 : (size_t)p.npts * 8;  // weights / offsets
  b += (size_t)(p.nTheta + 2 * p.L + p.nphi) * (cb + 4);       // twiddles + permutations
  b += fft_scratch_elems(p) * cb;                              // long-FFT buffers
  if (p.adj_threads == 32) b += (size_t)p.nalm * 16 + (size_t)(p.lmax + 1) * 4;  // FP32 adjoint accumulator
  // small tables: rings, seeds, ring ranges, deconvolution, weights, work items (upper bounds)
  b += (size_t)p.nring * (sizeof(RingDev) + rb) + (size_t)(p.lmax + 1) * (sizeof(MSeed) + 4 * sizeof(int2));
  b += (size_t)(2 * p.L + 2 * p.M + 2) * rb;
  const size_t items = (size_t)(p.M + 1) * (2 + (size_t)p.nring / 32);  // items hold >= 32 rings, one per part
  b += items * (sizeof(RecItem) + sizeof(AdjItem));
  b += ((size_t)p.ntr * p.ntq + (size_t)p.npts / 2048 + 1) * sizeof(TileItem);
  if (p.prec == 32) b += ((size_t)p.ntr * p.ntq * p.TR + 1) * sizeof(int);  // per-row point offsets
  {  // recursion start states: per order and ring part at most one part-filled item
    const size_t scap = 32 * (size_t)p.syn_rpt, acap = 32 * (size_t)p.adj_rpt, sb = p.prec == 64 ? 36 : 20;
    b += (size_t)(p.M + 1) * ((p.nring + 2 * scap) * sb + 4 * (4 + (size_t)p.nring / 32));
    if (p.prec == 32) b += (size_t)(p.M + 1) * (p.nring + 2 * acap) * sb;
    // FP64 block adjoint: every active (ring, order) pair once (36 B), and per (ring part, ring
    // chunk, order) an offset and a start l (12 B)
    if (p.prec == 64) {
      const size_t cr = (size_t)p.adj_rpt * p.adj_threads, nch = (p.nring + cr - 1) / cr;
      b += (size_t)(p.M + 1) * ((size_t)p.nring * 36 + 2 * nch * 12);
    }
  }
  if (p.patch) {  // rotator, rotated a_lm, spin phases and the adjoint's rotated input
    b += rotator_bytes(p.lmax, p.prec) + 2 * (size_t)p.nalm * cb;
    if (p.spin > 0) b += 2 * (size_t)p.npts * cb;
  }
  return b;
}

void destroy(Plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  for (void* a : p->allocs) cudaFree(a);
  rotator_destroy(p->rot);
  for (auto& r : p->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : p->evpool) cudaEventDestroy(e);
  for (cudaEvent_t e : p->chunk_ev) cudaEventDestroy(e);
  if (p->copy_st) cudaStreamDestroy(p->copy_st);
  delete p;
}

// Seeds of the recursion per order m: Wigner's closed form at l0 = max(m, s), as log2 of
// N_l0 sqrt(C(2 l0, p1)) and the powers of the half-angle cosine and sine, for the columns
// d_{m,-s} (e1) and d_{m,s} (e2).
std::vector<MSeed> make_seeds(int lmax, int spin) {
  std::vector<MSeed> ms(lmax + 1);
  for (int m = 0; m <= lmax; ++m) {
    MSeed d;
    d.l0 = std::max(m, spin);
    if (m >= spin) {
      d.p1 = m - spin;
      d.q1 = m + spin;
      d.sign1 = d.sign2 = ((m + spin) & 1) ? -1 : 1;
    } else {
      d.p1 = spin - m;
      d.q1 = spin + m;
      d.sign1 = ((spin + m) & 1) ? -1 : 1;
      d.sign2 = 1;
    }
    const long double l0 = d.l0;
    const long double lb = 0.5L * (lgammal(2 * l0 + 1) - lgammal((long double)d.p1 + 1) - lgammal((long double)d.q1 + 1)) /
                           logl(2.0L);
    const long double ln = 0.5L * log2l((2 * l0 + 1) / (4.0L * 3.14159265358979323846264338327950288L));
    d.lbin = (double)(lb + ln);
    ms[m] = d;
  }
  return ms;
}

// options in a plan, validated
void apply_options(Plan& p, const psht_options* opt) {
  if (!opt) return;
  PSHT_REQUIRE(opt->window == PSHT_WINDOW_ES || opt->window == PSHT_WINDOW_KB, PSHT_EINVAL, "unknown window");
  PSHT_REQUIRE(opt->kappa == 0.0 || (opt->kappa >= 0.25 && opt->kappa <= 4.0), PSHT_EINVAL,
               "kappa must be 0 (default) or lie in [0.25, 4]");
  PSHT_REQUIRE(opt->apodisation == PSHT_APO_PAPER || opt->apodisation == PSHT_APO_COST, PSHT_EINVAL,
               "unknown apodisation choice");
  p.window = opt->window;
  p.kappa = opt->kappa == 0.0 ? 1.0 : opt->kappa;
  p.apo_cost = opt->apodisation == PSHT_APO_COST ? 1 : 0;
}

// device scratch freed on scope exit (after the stream work that uses it: cudaFree waits for the device)
struct DevTmp {
  void* p = nullptr;
  ~DevTmp() {
    if (p) cudaFree(p);
  }
};

Plan* create(int spin, int lmax, const double* theta, const double* phi, int64_t npts, double eps, uint32_t flags,
             const psht_options* opt, cudaStream_t st) {
  PSHT_REQUIRE(spin >= 0, PSHT_EINVAL, "spin must be >= 0");
  PSHT_REQUIRE(lmax >= spin, PSHT_EINVAL, "lmax must be >= spin");
  PSHT_REQUIRE(lmax <= 65535, PSHT_EINVAL, "lmax above 65535");
  PSHT_REQUIRE(eps >= 1e-14 && eps <= 1e-1, PSHT_EINVAL, "eps must lie in [1e-14, 1e-1]");
  PSHT_REQUIRE(npts >= 0 && npts < ((int64_t)1 << 31), PSHT_EINVAL, "npts must lie in [0, 2^31)");
  PSHT_REQUIRE(npts == 0 || (theta && phi), PSHT_EINVAL, "theta and phi must be device pointers");
  const uint32_t pf = flags & 3u;
  PSHT_REQUIRE(pf != 3u, PSHT_EINVAL, "PSHT_FP32 and PSHT_FP64 are exclusive");
  PSHT_REQUIRE((flags & ~15u) == 0u, PSHT_EINVAL, "unknown flag bits");
  int prec = (pf == PSHT_FP64) ? 64 : (pf == PSHT_FP32) ? 32 : (eps >= 1e-5 ? 32 : 64);
  // FP64 everywhere below eps = 1e-6: the FP32 form's recursion and interpolation errors (a few
  // 1e-6 relative at lmax 4096-16384) would exceed the requested tolerance there
  PSHT_REQUIRE(!(prec == 32 && eps < 1e-6), PSHT_EINVAL, "the FP32 form needs eps >= 1e-6");

  Plan* p = new Plan();
  try {
    p->spin = spin;
    p->lmax = lmax;
    p->eps = eps;
    p->prec = prec;
    p->npts = npts;
    p->force_full = (flags & PSHT_FULL_SKY) ? 1 : 0;
    apply_options(*p, opt);
    // patch-centred frame: validate the caller's points, then rotate them (and keep each one's
    // spin-basis angle)
    DevTmp rpts;
    if (flags & PSHT_PATCH_FRAME) {
      p->patch = 1;
      if (npts > 0) {
        double red0[3];
        reduce_points(theta, phi, npts, red0, st);
        PSHT_REQUIRE(red0[2] == 0.0, PSHT_EINVAL, "theta outside [0, pi], NaN, or non-finite phi in the points");
        patch_rotation_device(theta, phi, npts, p->euler, nullptr, st);
        PSHT_CUDA_TRY(cudaMalloc(&rpts.p, (size_t)npts * 3 * sizeof(double)));
        double* t2 = (double*)rpts.p;
        rotate_points_device(p->euler[0], p->euler[1], p->euler[2], theta, phi, npts, t2, t2 + npts,
                             spin > 0 ? t2 + 2 * npts : nullptr, st);
        theta = t2;
        phi = t2 + npts;
      }
    }
    // step 1: nearer pole and theta* (one device reduction, validates the points)
    double red[3];
    reduce_points(theta, phi, npts, red, st);
    PSHT_REQUIRE(red[2] == 0.0, PSHT_EINVAL, "theta outside [0, pi], NaN, or non-finite phi in the points");
    p->pole = (red[0] <= red[1]) ? 1 : -1;
    layout(*p, p->pole > 0 ? red[0] : red[1]);

    // ring table
    // A ring at colatitude theta_j > pi/2 is evaluated at pi - theta_j by the reflection
    // d^l_{m,-s}(pi - b) = (-1)^(l+m) d^l_{m,s}(b), so every recurrence runs at b <= pi/2.
    std::vector<RingDev> rings(p->nring);
    std::vector<int> refl(p->nring);
    for (int j = 0; j < p->nring; ++j) {
      const double bj = p->beta_j[j];
      const double b = bj <= 0.5 * M_PI ? bj : M_PI - bj;
      refl[j] = p->pole > 0 ? (bj > 0.5 * M_PI) : (bj < 0.5 * M_PI);
      p->has_refl |= refl[j];
      RingDev r;
      const double sb = sin(0.5 * b), ch = cos(0.5 * b);
      r.omx = 2.0 * sb * sb;
      r.l2c = ch > 0 ? log2(ch) : -INFINITY;
      r.l2s = sb > 0 ? log2(sb) : -INFINITY;
      r.ohi = (float)r.omx;
      r.olo = (float)(r.omx - (double)r.ohi);
      rings[j] = r;
    }
    p->d_ring = (RingDev*)upload(*p, rings, st);
    // per-m seeds
    const std::vector<MSeed> ms = make_seeds(lmax, spin);
    p->d_mseed = (MSeed*)upload(*p, ms, st);
    // active ring ranges and synthesis work items
    // per order m and ring part (0: direct, 1: reflected) the active rings M_j >= m form one
    // contiguous range (M_j is unimodal in j, the reflection flag monotone)
    std::vector<int2> mr(2 * (size_t)(lmax + 1), make_int2(0, 0));
    for (int m = 0; m <= p->M; ++m) {
      for (int part = 0; part < 2; ++part) {
        int lo = -1, hi = -1;
        for (int j = 0; j < p->nring; ++j)
          if (p->Mj[j] >= m && refl[j] == part) {
            if (lo < 0) lo = j;
            hi = j + 1;
          }
        if (lo < 0) continue;
        mr[(size_t)part * (lmax + 1) + m] = make_int2(lo, hi);
        p->pairs += hi - lo;
        p->triples += (int64_t)(hi - lo) * (lmax - std::max(m, spin) + 1);
      }
    }
    // Mirror pairs (full-sky plans): ring jm - j lies at pi - b_j, so by d^l_{m,-s}(pi - b) =
    // (-1)^(l+m) d^l_{m,s}(b) it shares the Wigner columns of ring j.  An order whose reflected
    // active rings are exactly the mirrors of its direct ones (the equator ring, its own mirror,
    // aside) evaluates the columns once per pair.  pair[m] = the paired direct rings [a, b), eq[m] =
    // the equator ring when it is active and unpaired (else -1).
    const int jm = p->nring - 1;
    std::vector<int2> pair(lmax + 1, make_int2(0, 0));
    std::vector<int> eqr(lmax + 1, -1), mmode(lmax + 1, 0);
    bool any_mirror = false;
    if (p->full && p->has_refl) {
      const int eq = (jm % 2 == 0) ? jm / 2 : -1;
      for (int m = 0; m <= p->M; ++m) {
        const int2 D = mr[m], R = mr[(size_t)(lmax + 1) + m];
        if (D.y <= D.x || R.y <= R.x) continue;
        const int a = jm - (R.y - 1), b = jm - R.x + 1;  // mirror of the reflected range
        int e = -1;
        bool ok = (D.x == a && D.y == b);
        if (!ok && eq >= 0 && D.x == a && D.y == b + 1 && b == eq) ok = true, e = eq;
        if (!ok && eq >= 0 && D.x == a - 1 && D.y == b && a - 1 == eq) ok = true, e = eq;
        if (!ok || refl[a] != 0) continue;
        pair[m] = make_int2(a, b);
        eqr[m] = e;
        mmode[m] = 1;
        any_mirror = true;
      }
    }
    std::vector<RecItem> items, mitems;
    const int cap = p->syn_rpt * p->syn_threads;
    auto chunks = [](int lo, int hi, int cp, auto&& emit) {
      const int n = hi - lo, nchunk = (n + cp - 1) / cp;
      for (int c = 0; c < nchunk; ++c)
        emit(lo + (int)((int64_t)n * c / nchunk), lo + (int)((int64_t)n * (c + 1) / nchunk));
    };
    for (int m = 0; m <= p->M; ++m) {
      if (mmode[m]) {
        chunks(pair[m].x, pair[m].y, cap, [&](int a, int b) { mitems.push_back(RecItem{m, a, b - a, 0}); });
        if (eqr[m] >= 0) items.push_back(RecItem{m, eqr[m], 1, 0});
        continue;
      }
      for (int part = 0; part < 2; ++part) {
        const int2 r = mr[(size_t)part * (lmax + 1) + m];
        if (r.y > r.x) chunks(r.x, r.y, cap, [&](int a, int b) { items.push_back(RecItem{m, a, b - a, part}); });
      }
    }
    p->d_mrange = (int2*)upload(*p, mr, st);
    p->nitems = (int)items.size();
    p->d_items = (RecItem*)upload(*p, items, st);
    p->nmitems = (int)mitems.size();
    if (p->nmitems > 0) p->d_mitems = (RecItem*)upload(*p, mitems, st);
    if (any_mirror && prec == 64) p->d_mmode = (int*)upload(*p, mmode, st);
    if (p->adj_threads == 32) {  // one-warp adjoint: items of at most 32 adj_rpt rings, per-m spans
      const int acap = 32 * p->adj_rpt;
      std::vector<AdjItem> ai, mai;
      std::vector<int2> span(lmax + 1, make_int2(0, 0));  // .y: items of order m (both lists)
      for (int m = 0; m <= p->M; ++m) {
        span[m].x = (int)ai.size();
        if (mmode[m]) {
          chunks(pair[m].x, pair[m].y, acap, [&](int a, int b) { mai.push_back(AdjItem{m, a, b - a, 0, 0}); });
          if (eqr[m] >= 0) ai.push_back(AdjItem{m, eqr[m], 1, 0, 0});
        } else {
          for (int part = 0; part < 2; ++part) {
            const int2 r = mr[(size_t)part * (lmax + 1) + m];
            if (r.y > r.x)
              chunks(r.x, r.y, acap, [&](int a, int b) { ai.push_back(AdjItem{m, a, b - a, part, 0}); });
          }
        }
      }
      for (const AdjItem& x : ai) ++span[x.m].y;
      for (const AdjItem& x : mai) ++span[x.m].y;
      for (AdjItem& x : ai) x.nitems = span[x.m].y;
      for (AdjItem& x : mai) x.nitems = span[x.m].y;
      p->naitems = (int)ai.size();
      p->d_aitems = ai.empty() ? nullptr : (AdjItem*)upload(*p, ai, st);
      p->nmaitems = (int)mai.size();
      if (p->nmaitems > 0) p->d_maitems = (AdjItem*)upload(*p, mai, st);
      p->d_aspan = (int2*)upload(*p, span, st);
      // accumulator and arrival counters start at zero; every call leaves them at zero
      p->d_acc = dalloc(*p, (size_t)p->nalm * 16);
      p->d_cnt = (int*)dalloc(*p, (size_t)(lmax + 1) * sizeof(int));
      PSHT_CUDA_TRY(cudaMemsetAsync(p->d_acc, 0, (size_t)p->nalm * 16, st));
      PSHT_CUDA_TRY(cudaMemsetAsync(p->d_cnt, 0, (size_t)(lmax + 1) * sizeof(int), st));
      // order chunks for the host-buffer entry points, split at order boundaries by recursion
      // work (ring count x l range of the items): the synthesis in 10 / 30 / 60 % of its work, so
      // that only the first tenth of the a_lm upload is not hidden behind a recursion launch (the
      // upload of a part takes about a third of its recursion's time); the adjoint in 60 / 30 /
      // 10 %, so that only the last tenth of the download follows the last launch.  Three launches
      // each: every launch adds its tail (its longest warps), so few chunks beat many.  Plans with
      // mirror pairs run unchunked (no chunk table).
      if (!any_mirror) {
        const auto split = [&](const auto& its, std::initializer_list<double> fr, std::vector<int>& cm,
                               std::vector<int>& ci) {
          std::vector<double> cum(its.size() + 1, 0.0);
          for (size_t i = 0; i < its.size(); ++i)
            cum[i + 1] = cum[i] + (double)its[i].nj * (lmax - std::max(its[i].m, spin) + 1);
          cm.assign(1, 0);
          for (double f : fr) {
            const size_t i = std::lower_bound(cum.begin(), cum.end(), cum.back() * f) - cum.begin();
            if (i >= its.size()) break;
            if (its[i].m > cm.back()) cm.push_back(its[i].m);
          }
          cm.push_back(p->M + 1);
          for (int mb : cm) {
            int it = 0;
            while (it < (int)its.size() && its[it].m < mb) ++it;
            ci.push_back(it);
          }
        };
        split(items, {0.1, 0.4}, p->chunk_m, p->chunk_item);
        split(ai, {0.6, 0.9}, p->achunk_m, p->chunk_aitem);
      }
    }
    // deconvolution tables, ring weights, FFT twiddles and digit-reversal tables
    static const Quad quad;
    std::vector<double> sT(2 * p->L - 1), sP(2 * p->M + 1);
    const double hT = 2.0 * M_PI / p->nTheta, hP = 2.0 * M_PI / p->nphi;
    for (int i = 0; i < 2 * p->L - 1; ++i)
      sT[i] = hT / (2.0 * p->L * es_ft(i - (p->L - 1), p->W, p->beta_es, p->nTheta, quad));
    for (int i = 0; i < 2 * p->M + 1; ++i) sP[i] = hP / es_ft(i - p->M, p->W, p->beta_es, p->nphi, quad);
    p->f2L = radix_schedule(2 * p->L);
    p->f4L = radix_schedule(4 * p->L);
    p->fP = radix_schedule(p->nphi);
    p->d_perm2L = (int*)upload(*p, fft_perm(p->f2L), st);
    p->d_perm4L = (int*)upload(*p, fft_perm(p->f4L), st);
    p->d_permP = (int*)upload(*p, fft_perm(p->fP), st);
    auto twid = [](int n) {
      std::vector<double> t(2 * (size_t)n);
      for (int k = 0; k < n; ++k) {
        const double a = 2.0 * M_PI * k / n;
        t[2 * k] = cos(a);
        t[2 * k + 1] = -sin(a);
      }
      return t;
    };
    // FP32 form: e^{-2 pi i t/n} as tw[t & 63] tw[64 + (t >> 6)], the 64 fine and n/64 + 1 coarse
    // factors (psht_common.cuh, twiddle<float2>)
    auto twid_split = [](int n) {
      const int nb = n / 64 + 1;
      std::vector<double> t(2 * (size_t)(64 + nb));
      for (int k = 0; k < 64 + nb; ++k) {
        const double a = 2.0 * M_PI * (k < 64 ? k : 64.0 * (k - 64)) / n;
        t[2 * k] = cos(a);
        t[2 * k + 1] = -sin(a);
      }
      return t;
    };
    if (prec == 64) {
      p->d_sT = upload(*p, sT, st);
      p->d_sP = upload(*p, sP, st);
      p->d_w = upload(*p, p->w_j, st);
      p->d_tw2L = upload(*p, twid(2 * p->L), st);
      p->d_tw4L = upload(*p, twid(4 * p->L), st);
      p->d_twP = upload(*p, twid(p->nphi), st);
    } else {
      p->d_sT = upload(*p, cast_vec<float>(sT), st);
      p->d_sP = upload(*p, cast_vec<float>(sP), st);
      p->d_w = upload(*p, cast_vec<float>(p->w_j), st);
      p->d_tw2L = upload(*p, cast_vec<float>(twid_split(2 * p->L)), st);
      p->d_tw4L = upload(*p, cast_vec<float>(twid_split(4 * p->L)), st);
      p->d_twP = upload(*p, cast_vec<float>(twid_split(p->nphi)), st);
    }
    // work buffers
    const size_t cb = prec == 64 ? 16 : 8;
    p->d_rtab = dalloc(*p, (size_t)rec_table_record_bytes(p->prec) * p->tstride);
    PSHT_CUDA_TRY(cudaMemsetAsync(p->d_rtab, 0, (size_t)rec_table_record_bytes(p->prec) * p->tstride, st));
    p->d_status = (int*)dalloc(*p, sizeof(int));
    PSHT_CUDA_TRY(cudaMemsetAsync(p->d_status, 0, sizeof(int), st));
    p->d_F = dalloc(*p, (size_t)p->ncols * p->Lpad * cb);
    p->d_X = dalloc(*p, (size_t)p->nrows * p->ncols * cb);
    p->d_G = dalloc(*p, (size_t)p->nrows * p->gstride * cb);
    if (const size_t fe = fft_scratch_elems(*p)) p->d_fscratch = dalloc(*p, fe * cb);
    build_rec_table(*p, st);
    {  // start states of the one-warp recursion items (after the table they are stepped with)
      const size_t sb = 4 * (size_t)(prec == 64 ? 8 : 4);  // (e1, d1, e2, d2) per slot
      const auto alloc_start = [&](RecStart& r, int n, int slots) {
        if (n <= 0) return;
        r.ls = (int*)dalloc(*p, (size_t)n * sizeof(int));
        r.st = dalloc(*p, (size_t)n * slots * sb);
        r.kk = (int*)dalloc(*p, (size_t)n * slots * sizeof(int));
      };
      alloc_start(p->s_items, p->nitems, 32 * p->syn_rpt);
      alloc_start(p->s_mitems, p->nmitems, 32 * p->syn_rpt);
      if (prec == 32) {
        alloc_start(p->s_aitems, p->naitems, 32 * p->adj_rpt);
        alloc_start(p->s_maitems, p->nmaitems, 32 * p->adj_rpt);
      } else {  // FP64 block adjoint: per (ring part, ring chunk, order) the chunk's active rings
        const int cr = p->adj_rpt * p->adj_threads, nch = (p->nring + cr - 1) / cr;
        const int nparts = p->has_refl ? 2 : 1;
        std::vector<int64_t> off((size_t)nparts * nch * (p->M + 1));
        int64_t tot = 0;
        for (int part = 0; part < nparts; ++part)
          for (int chk = 0; chk < nch; ++chk)
            for (int m = 0; m <= p->M; ++m) {
              off[((size_t)part * nch + chk) * (p->M + 1) + m] = tot;
              const int2 r = mr[(size_t)part * (lmax + 1) + m];
              const int a = r.x + chk * cr, b = std::min(r.y, a + cr);
              tot += std::max(0, b - a);
            }
        p->badj_nch = nch;
        p->s_badj_off = (int64_t*)upload(*p, off, st);
        p->s_badj.ls = (int*)dalloc(*p, off.size() * sizeof(int));
        p->s_badj.st = dalloc(*p, (size_t)std::max<int64_t>(tot, 1) * 4 * sizeof(double));
        p->s_badj.kk = (int*)dalloc(*p, (size_t)std::max<int64_t>(tot, 1) * sizeof(int));
      }
      build_rec_starts(*p, st);
    }
    // step 3 for the points: Theta_p, tiles, sorted layout (and FP64 kernel weights)
    if (prec == 64) {
      p->d_pidx = (int32_t*)dalloc(*p, (size_t)std::max<int64_t>(npts, 1) * 4);
      p->d_pcell = (int32_t*)dalloc(*p, (size_t)std::max<int64_t>(npts, 1) * 4);
      p->d_pw = dalloc(*p, (size_t)std::max<int64_t>(npts, 1) * 2 * p->W * 8);
    } else {  // one 16-byte record per point: a single load per point in the spreading kernel
      p->d_prec = (int4*)dalloc(*p, (size_t)std::max<int64_t>(npts, 1) * sizeof(int4));
    }
    bin_points(*p, theta, phi, st);
    if (p->patch) {
      p->rot = rotator_create(lmax, prec, st);
      p->bytes += rotator_bytes(lmax, prec);
      p->d_ra = dalloc(*p, 2 * (size_t)p->nalm * cb);
      if (spin > 0 && npts > 0) {
        p->d_sph = dalloc(*p, (size_t)npts * cb);
        p->d_fr = dalloc(*p, (size_t)npts * cb);
        spin_phase_device(prec, (const double*)rpts.p + 2 * npts, spin, npts, p->d_sph, st);
      }
    }
    PSHT_CUDA_TRY(cudaStreamSynchronize(st));
    return p;
  } catch (...) {
    destroy(p);
    throw;
  }
}

int fail(const Error& e) {
  set_error(e.msg);
  return e.code;
}

template <class F>
int guarded(F&& f) {
  try {
    g_err.clear();
    f();
    return PSHT_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::bad_alloc&) {
    return fail(Error{PSHT_ENOMEM, "host allocation failed"});
  } catch (...) {
    return fail(Error{PSHT_ECUDA, "unexpected failure"});
  }
}

cudaEvent_t take_event(Plan& p) {
  if (!p.evpool.empty()) {
    cudaEvent_t e = p.evpool.back();
    p.evpool.pop_back();
    return e;
  }
  cudaEvent_t e;
  PSHT_CUDA_TRY(cudaEventCreate(&e));
  return e;
}

// run fn() as stage `stage`, bracketed by events when profiling is on
template <class F>
void staged(Plan& p, int stage, cudaStream_t st, F&& fn) {
  if (!p.profile) {
    fn();
    return;
  }
  Plan::StageRec r{stage, take_event(p), take_event(p)};
  PSHT_CUDA_TRY(cudaEventRecord(r.a, st));
  fn();
  PSHT_CUDA_TRY(cudaEventRecord(r.b, st));
  p.recs.push_back(r);
}

void run_synthesis(Plan& p, const void* g, const void* c, void* f, cudaStream_t st, double msc = 1.0) {
  staged(p, 0, st, [&] { launch_rec_synthesis(p, g, c, st, msc); });
  staged(p, 1, st, [&] { launch_theta_synthesis(p, st); });
  staged(p, 2, st, [&] { launch_phi_synthesis(p, st); });
  staged(p, 3, st, [&] { launch_gather(p, f, st); });
}

void run_adjoint(Plan& p, const void* f, void* g, void* c, cudaStream_t st, double msc = 1.0) {
  const size_t cb = p.prec == 64 ? 16 : 8;
  staged(p, 4, st, [&] {
    PSHT_CUDA_TRY(cudaMemsetAsync(p.d_G, 0, (size_t)p.nrows * p.gstride * cb, st));
    launch_scatter(p, f, st);
  });
  staged(p, 5, st, [&] { launch_phi_adjoint(p, st); });
  staged(p, 6, st, [&] { launch_theta_adjoint(p, st); });
  staged(p, 7, st, [&] { launch_rec_adjoint(p, g, c, st, msc); });
}

// Batched execution: groups of up to kBatchGroup sets share one recursion launch (the Wigner
// columns are evaluated once per (ring, m, l) for the whole group); the FFT, gather and scatter
// stages run per set on the group's own ring-coefficient buffers.
constexpr int kBatchGroup = 4;

void ensure_batch(Plan& p, int nsets, cudaStream_t st) {
  const int need = std::min(nsets, kBatchGroup) - 1;
  const size_t cb = p.prec == 64 ? 16 : 8;
  while ((int)p.d_Fb.size() < need) {
    p.d_Fb.push_back(dalloc(p, (size_t)p.ncols * p.Lpad * cb));
    if (p.adj_threads == 32) {  // FP32 adjoint accumulator of the extra set (zero between calls)
      void* a = dalloc(p, (size_t)p.nalm * 16);
      PSHT_CUDA_TRY(cudaMemsetAsync(a, 0, (size_t)p.nalm * 16, st));
      p.d_accb.push_back(a);
    } else {
      p.d_accb.push_back(nullptr);
    }
  }
}

void run_synthesis_batch(Plan& p, int nsets, const void* const* g, const void* const* c, void* const* f,
                         cudaStream_t st, double msc = 1.0) {
  ensure_batch(p, nsets, st);
  void* const F0 = p.d_F;
  for (int k0 = 0; k0 < nsets; k0 += kBatchGroup) {
    const int n = std::min(kBatchGroup, nsets - k0);
    void* Fs[kBatchGroup] = {F0};
    for (int k = 1; k < n; ++k) Fs[k] = p.d_Fb[k - 1];
    staged(p, 0, st, [&] { launch_rec_synthesis_sets(p, n, g + k0, c ? c + k0 : nullptr, Fs, st, msc); });
    try {
      for (int k = 0; k < n; ++k) {
        p.d_F = Fs[k];
        staged(p, 1, st, [&] { launch_theta_synthesis(p, st); });
        staged(p, 2, st, [&] { launch_phi_synthesis(p, st); });
        staged(p, 3, st, [&] { launch_gather(p, f[k0 + k], st); });
      }
    } catch (...) {
      p.d_F = F0;
      throw;
    }
    p.d_F = F0;
  }
}

void run_adjoint_batch(Plan& p, int nsets, const void* const* f, void* const* g, void* const* c, cudaStream_t st,
                       double msc = 1.0) {
  ensure_batch(p, nsets, st);
  const size_t cb = p.prec == 64 ? 16 : 8;
  void* const F0 = p.d_F;
  for (int k0 = 0; k0 < nsets; k0 += kBatchGroup) {
    const int n = std::min(kBatchGroup, nsets - k0);
    void* Fs[kBatchGroup] = {F0};
    void* accs[kBatchGroup] = {p.d_acc};
    for (int k = 1; k < n; ++k) {
      Fs[k] = p.d_Fb[k - 1];
      accs[k] = p.d_accb[k - 1];
    }
    try {
      for (int k = 0; k < n; ++k) {
        staged(p, 4, st, [&] {
          PSHT_CUDA_TRY(cudaMemsetAsync(p.d_G, 0, (size_t)p.nrows * p.gstride * cb, st));
          launch_scatter(p, f[k0 + k], st);
        });
        staged(p, 5, st, [&] { launch_phi_adjoint(p, st); });
        p.d_F = Fs[k];
        staged(p, 6, st, [&] { launch_theta_adjoint(p, st); });
        p.d_F = F0;
      }
    } catch (...) {
      p.d_F = F0;
      throw;
    }
    staged(p, 7, st, [&] { launch_rec_adjoint_sets(p, n, Fs, accs, g + k0, c ? c + k0 : nullptr, st, msc); });
  }
}

// Synthesis and adjoint as the entry points see them: in a patch-frame plan the a_lm are rotated
// into the plan's frame first (the synthesis weight msc applies to the caller's m > 0 entries), and
// the spin-s values carry each point's basis angle, f(p) = e^{i s psi_p} f'(R p); the adjoint is
// the exact transpose: conjugate phase, adjoint in the plan's frame, inverse rotation.
// rotate = false: the a_lm are already in the plan's frame (PSHT_PATCH_FRAME plans only)
void exec_synthesis(Plan& p, const void* g, const void* c, void* f, cudaStream_t st, double msc = 1.0,
                    bool rotate = true) {
  if (!p.patch) {
    run_synthesis(p, g, c, f, st, msc);
    return;
  }
  if (!rotate) {
    run_synthesis(p, g, c, f, st, msc);
    if (p.d_sph) mul_phase_device(p.prec, f, p.d_sph, p.npts, false, f, st);
    return;
  }
  const size_t na = (size_t)p.nalm * (p.prec == 64 ? 16 : 8);
  char* ra = (char*)p.d_ra;
  rotator_apply(*p.rot, p.euler[0], p.euler[1], p.euler[2], g, c, ra, c ? ra + na : nullptr, st, msc, 1.0);
  run_synthesis(p, ra, c ? ra + na : nullptr, f, st);
  if (p.d_sph) mul_phase_device(p.prec, f, p.d_sph, p.npts, false, f, st);
}

void exec_adjoint(Plan& p, const void* f, void* g, void* c, cudaStream_t st, double msc = 1.0, bool rotate = true) {
  if (!p.patch) {
    run_adjoint(p, f, g, c, st, msc);
    return;
  }
  const size_t na = (size_t)p.nalm * (p.prec == 64 ? 16 : 8);
  char* ra = (char*)p.d_ra;
  const void* fr = f;
  if (p.d_sph) {
    mul_phase_device(p.prec, f, p.d_sph, p.npts, true, p.d_fr, st);
    fr = p.d_fr;
  }
  if (!rotate) {
    run_adjoint(p, fr, g, c, st, msc);
    return;
  }
  run_adjoint(p, fr, ra, c ? ra + na : nullptr, st);
  rotator_apply(*p.rot, -p.euler[2], -p.euler[1], -p.euler[0], ra, c ? ra + na : nullptr, g, c, st, 1.0, msc);
}

void ensure_io(Plan& p) {
  const size_t cb = p.prec == 64 ? 16 : 8;
  if (!p.d_io_a) p.d_io_a = dalloc(p, 2 * (size_t)p.nalm * cb);
  if (!p.d_io_f) p.d_io_f = dalloc(p, (size_t)std::max<int64_t>(p.npts, 1) * cb);
  if (!p.chunk_m.empty() && !p.copy_st) {
    PSHT_CUDA_TRY(cudaStreamCreateWithFlags(&p.copy_st, cudaStreamNonBlocking));
    p.chunk_ev.resize(std::max(p.chunk_m.size(), p.achunk_m.size()) + 1);
    for (auto& e : p.chunk_ev) PSHT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
}

// resets the plan's launch ranges on scope exit, also when a launch throws
struct RangeReset {
  Plan& p;
  ~RangeReset() {
    p.r_item0 = p.r_aitem0 = p.r_m0 = 0;
    p.r_item1 = p.r_aitem1 = p.r_m1 = -1;
  }
};

// first packed index of order m (orders m' < m hold lmax - m' + 1 entries each); nalm at m = lmax + 1
int64_t alm_off(int lmax, int m) { return (int64_t)m * (2 * lmax + 3 - m) / 2; }

// Host-buffer synthesis with the a_lm upload overlapping the recursion: the orders of chunk k are
// copied on the copy stream and the recursion items of those orders start as soon as they landed.
void synthesis_host_chunked(Plan& p, const void* g, const void* c, void* f, cudaStream_t st) {
  const size_t cb = p.prec == 64 ? 16 : 8, na = (size_t)p.nalm * cb;
  char* da = (char*)p.d_io_a;
  const int K = (int)p.chunk_m.size() - 1;
  cudaEvent_t start = p.chunk_ev[K];
  PSHT_CUDA_TRY(cudaEventRecord(start, st));  // earlier work on st may still read the staging
  PSHT_CUDA_TRY(cudaStreamWaitEvent(p.copy_st, start, 0));
  for (int k = 0; k < K; ++k) {
    const size_t b0 = alm_off(p.lmax, p.chunk_m[k]) * cb, b1 = alm_off(p.lmax, p.chunk_m[k + 1]) * cb;
    PSHT_CUDA_TRY(cudaMemcpyAsync(da + b0, (const char*)g + b0, b1 - b0, cudaMemcpyHostToDevice, p.copy_st));
    if (c) PSHT_CUDA_TRY(cudaMemcpyAsync(da + na + b0, (const char*)c + b0, b1 - b0, cudaMemcpyHostToDevice, p.copy_st));
    PSHT_CUDA_TRY(cudaEventRecord(p.chunk_ev[k], p.copy_st));
  }
  RangeReset reset{p};
  staged(p, 0, st, [&] {
    for (int k = 0; k < K; ++k) {
      PSHT_CUDA_TRY(cudaStreamWaitEvent(st, p.chunk_ev[k], 0));
      p.r_item0 = p.chunk_item[k];
      p.r_item1 = p.chunk_item[k + 1];
      launch_rec_synthesis(p, da, c ? da + na : nullptr, st);
    }
    p.r_item0 = 0;
    p.r_item1 = -1;
  });
  staged(p, 1, st, [&] { launch_theta_synthesis(p, st); });
  staged(p, 2, st, [&] { launch_phi_synthesis(p, st); });
  staged(p, 3, st, [&] { launch_gather(p, p.d_io_f, st); });
  PSHT_CUDA_TRY(cudaMemcpyAsync(f, p.d_io_f, (size_t)p.npts * cb, cudaMemcpyDeviceToHost, st));
}

// Host-buffer adjoint with the download overlapping the recursion: after the recursion items and
// the reduction of the orders of chunk k, their g~ and c~ go to the host on the copy stream.
void adjoint_host_chunked(Plan& p, const void* f, void* g, void* c, cudaStream_t st) {
  const size_t cb = p.prec == 64 ? 16 : 8, na = (size_t)p.nalm * cb;
  char* da = (char*)p.d_io_a;
  const int K = (int)p.achunk_m.size() - 1;
  PSHT_CUDA_TRY(cudaMemcpyAsync(p.d_io_f, f, (size_t)p.npts * cb, cudaMemcpyHostToDevice, st));
  staged(p, 4, st, [&] {
    PSHT_CUDA_TRY(cudaMemsetAsync(p.d_G, 0, (size_t)p.nrows * p.gstride * cb, st));
    launch_scatter(p, p.d_io_f, st);
  });
  staged(p, 5, st, [&] { launch_phi_adjoint(p, st); });
  staged(p, 6, st, [&] { launch_theta_adjoint(p, st); });
  RangeReset reset{p};
  staged(p, 7, st, [&] {
    for (int k = 0; k < K; ++k) {
      p.r_aitem0 = p.chunk_aitem[k];
      p.r_aitem1 = p.chunk_aitem[k + 1];
      p.r_m0 = p.achunk_m[k];
      p.r_m1 = k + 1 < K ? p.achunk_m[k + 1] : p.lmax + 1;  // the last chunk also writes the zero orders
      launch_rec_adjoint(p, da, c ? da + na : nullptr, st);
      PSHT_CUDA_TRY(cudaEventRecord(p.chunk_ev[k], st));
      PSHT_CUDA_TRY(cudaStreamWaitEvent(p.copy_st, p.chunk_ev[k], 0));
      const size_t b0 = alm_off(p.lmax, p.r_m0) * cb, b1 = alm_off(p.lmax, p.r_m1) * cb;
      PSHT_CUDA_TRY(cudaMemcpyAsync((char*)g + b0, da + b0, b1 - b0, cudaMemcpyDeviceToHost, p.copy_st));
      if (c) PSHT_CUDA_TRY(cudaMemcpyAsync((char*)c + b0, da + na + b0, b1 - b0, cudaMemcpyDeviceToHost, p.copy_st));
    }
    p.r_aitem0 = 0;
    p.r_aitem1 = -1;
    p.r_m0 = 0;
    p.r_m1 = -1;
  });
  PSHT_CUDA_TRY(cudaEventRecord(p.chunk_ev[K], p.copy_st));
  PSHT_CUDA_TRY(cudaStreamWaitEvent(st, p.chunk_ev[K], 0));
}

}  // namespace
}  // namespace psht

using namespace psht;

extern "C" {

struct psht_plan {
  Plan* p;
};

int psht_plan_create(int spin, int lmax, const double* theta, const double* phi, int64_t npts, double eps,
                     uint32_t flags, void* stream, psht_plan** out) {
  return guarded([&] {
    PSHT_REQUIRE(out != nullptr, PSHT_EINVAL, "out must not be NULL");
    *out = nullptr;
    Plan* p = create(spin, lmax, theta, phi, npts, eps, flags, nullptr, (cudaStream_t)stream);
    *out = new psht_plan{p};
  });
}

int psht_plan_create_ex(int spin, int lmax, const double* theta, const double* phi, int64_t npts, double eps,
                        uint32_t flags, const psht_options* opt, void* stream, psht_plan** out) {
  return guarded([&] {
    PSHT_REQUIRE(out != nullptr, PSHT_EINVAL, "out must not be NULL");
    *out = nullptr;
    Plan* p = create(spin, lmax, theta, phi, npts, eps, flags, opt, (cudaStream_t)stream);
    *out = new psht_plan{p};
  });
}

static void fill_info(const Plan& p, psht_info* info) {
    psht_info i;
    memset(&i, 0, sizeof(i));
    i.spin = p.spin;
    i.lmax = p.lmax;
    i.precision = p.prec;
    i.pole = p.pole;
    i.full_sky = p.full;
    i.eps = p.eps;
    i.theta_star = p.theta_star;
    i.eps_apo = p.eps_apo;
    i.theta_max = p.theta_max;
    i.alpha = p.alpha;
    i.dTheta = p.dTheta;
    i.Lmax = p.Lmax;
    i.L = p.L;
    i.nring = p.nring;
    i.M = p.M;
    i.W = p.W;
    i.beta_es = p.beta_es;
    i.nTheta = p.nTheta;
    i.nphi = p.nphi;
    i.r_lo = p.r_lo;
    i.nrows = p.nrows;
    i.npts = p.npts;
    i.ring_mode_pairs = p.pairs;
    i.recursion_triples = p.triples;
    i.device_bytes = p.bytes;
    i.patch_frame = p.patch;
    for (int k = 0; k < 3; ++k) i.euler[k] = p.euler[k];
    *info = i;
}

int psht_plan_info(const psht_plan* plan, psht_info* info) {
  return guarded([&] {
    PSHT_REQUIRE(plan && info, PSHT_EINVAL, "plan and info must not be NULL");
    fill_info(*plan->p, info);
  });
}

int psht_plan_params(int spin, int lmax, double theta_star, double eps, uint32_t flags, const psht_options* opt,
                     psht_info* info, double* theta_j, double* w_j, int32_t* Mj) {
  return guarded([&] {
    PSHT_REQUIRE(info, PSHT_EINVAL, "info must not be NULL");
    PSHT_REQUIRE(spin >= 0 && lmax >= spin && lmax <= 65535, PSHT_EINVAL, "invalid spin or lmax");
    PSHT_REQUIRE(eps >= 1e-14 && eps <= 1e-1, PSHT_EINVAL, "eps must lie in [1e-14, 1e-1]");
    PSHT_REQUIRE(theta_star >= 0.0 && theta_star <= M_PI, PSHT_EINVAL, "theta_star must lie in [0, pi]");
    const uint32_t pf = flags & 3u;
    PSHT_REQUIRE(pf != 3u && (flags & ~15u) == 0u, PSHT_EINVAL, "invalid flags");
    Plan p;
    p.spin = spin;
    p.lmax = lmax;
    p.eps = eps;
    p.prec = (pf == PSHT_FP64) ? 64 : (pf == PSHT_FP32) ? 32 : (eps >= 1e-5 ? 32 : 64);
    p.force_full = (flags & PSHT_FULL_SKY) ? 1 : 0;
    p.patch = (flags & PSHT_PATCH_FRAME) ? 1 : 0;
    p.pole = 1;
    apply_options(p, opt);
    layout(p, theta_star);
    for (int j = 0; j < p.nring; ++j) {
      p.pairs += p.Mj[j] + 1;
      p.triples += ring_cost(p.lmax, p.spin, p.Mj[j]);
      if (theta_j) theta_j[j] = p.theta_j[j];
      if (w_j) w_j[j] = p.w_j[j];
      if (Mj) Mj[j] = p.Mj[j];
    }
    p.bytes = planned_bytes(p);
    fill_info(p, info);
  });
}

int psht_plan_synthesis(psht_plan* plan, const void* g, const void* c, void* f, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g, PSHT_EINVAL, "plan and g must not be NULL");
    PSHT_REQUIRE(f || plan->p->npts == 0, PSHT_EINVAL, "f must not be NULL");
    exec_synthesis(*plan->p, g, c, f, (cudaStream_t)stream);
  });
}

int psht_plan_adjoint(psht_plan* plan, const void* f, void* g, void* c, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g, PSHT_EINVAL, "plan and g must not be NULL");
    PSHT_REQUIRE(f || plan->p->npts == 0, PSHT_EINVAL, "f must not be NULL");
    exec_adjoint(*plan->p, f, g, c, (cudaStream_t)stream);
  });
}

int psht_plan_synthesis_batch(psht_plan* plan, int nsets, const void* const* g, const void* const* c, void* const* f,
                              void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g && f, PSHT_EINVAL, "plan, g and f must not be NULL");
    PSHT_REQUIRE(nsets >= 1 && nsets <= PSHT_MAX_BATCH, PSHT_EINVAL, "nsets must lie in [1, PSHT_MAX_BATCH]");
    Plan& p = *plan->p;
    for (int k = 0; k < nsets; ++k) {
      PSHT_REQUIRE(g[k], PSHT_EINVAL, "g[k] must not be NULL");
      PSHT_REQUIRE(f[k] || p.npts == 0, PSHT_EINVAL, "f[k] must not be NULL");
    }
    if (p.patch) {  // the rotation works on one set at a time
      for (int k = 0; k < nsets; ++k) exec_synthesis(p, g[k], c ? c[k] : nullptr, f[k], (cudaStream_t)stream);
      return;
    }
    run_synthesis_batch(p, nsets, g, c, f, (cudaStream_t)stream);
  });
}
int psht_plan_adjoint_batch(psht_plan* plan, int nsets, const void* const* f, void* const* g, void* const* c,
                            void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g && f, PSHT_EINVAL, "plan, f and g must not be NULL");
    PSHT_REQUIRE(nsets >= 1 && nsets <= PSHT_MAX_BATCH, PSHT_EINVAL, "nsets must lie in [1, PSHT_MAX_BATCH]");
    Plan& p = *plan->p;
    for (int k = 0; k < nsets; ++k) {
      PSHT_REQUIRE(g[k], PSHT_EINVAL, "g[k] must not be NULL");
      PSHT_REQUIRE(f[k] || p.npts == 0, PSHT_EINVAL, "f[k] must not be NULL");
    }
    if (p.patch) {
      for (int k = 0; k < nsets; ++k) exec_adjoint(p, f[k], g[k], c ? c[k] : nullptr, (cudaStream_t)stream);
      return;
    }
    run_adjoint_batch(p, nsets, f, g, c, (cudaStream_t)stream);
  });
}

int psht_plan_synthesis_packed(psht_plan* plan, const void* g, const void* c, void* f, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g, PSHT_EINVAL, "plan and g must not be NULL");
    PSHT_REQUIRE(f || plan->p->npts == 0, PSHT_EINVAL, "f must not be NULL");
    exec_synthesis(*plan->p, g, c, f, (cudaStream_t)stream, 0.5);
  });
}

int psht_plan_adjoint_packed(psht_plan* plan, const void* f, void* g, void* c, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g, PSHT_EINVAL, "plan and g must not be NULL");
    PSHT_REQUIRE(f || plan->p->npts == 0, PSHT_EINVAL, "f must not be NULL");
    exec_adjoint(*plan->p, f, g, c, (cudaStream_t)stream, 2.0);
  });
}

int psht_plan_synthesis_inframe(psht_plan* plan, const void* g, const void* c, void* f, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g, PSHT_EINVAL, "plan and g must not be NULL");
    PSHT_REQUIRE(f || plan->p->npts == 0, PSHT_EINVAL, "f must not be NULL");
    PSHT_REQUIRE(plan->p->patch, PSHT_EINVAL, "the plan was not created with PSHT_PATCH_FRAME");
    exec_synthesis(*plan->p, g, c, f, (cudaStream_t)stream, 1.0, false);
  });
}

int psht_plan_adjoint_inframe(psht_plan* plan, const void* f, void* g, void* c, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g, PSHT_EINVAL, "plan and g must not be NULL");
    PSHT_REQUIRE(f || plan->p->npts == 0, PSHT_EINVAL, "f must not be NULL");
    PSHT_REQUIRE(plan->p->patch, PSHT_EINVAL, "the plan was not created with PSHT_PATCH_FRAME");
    exec_adjoint(*plan->p, f, g, c, (cudaStream_t)stream, 1.0, false);
  });
}

int psht_plan_synthesis_host(psht_plan* plan, const void* g, const void* c, void* f, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g && f, PSHT_EINVAL, "plan, g and f must not be NULL");
    Plan& p = *plan->p;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_io(p);
    const size_t cb = p.prec == 64 ? 16 : 8, na = (size_t)p.nalm * cb;
    char* da = (char*)p.d_io_a;
    if (!p.chunk_m.empty() && !p.patch) {
      synthesis_host_chunked(p, g, c, f, st);
    } else {
      PSHT_CUDA_TRY(cudaMemcpyAsync(da, g, na, cudaMemcpyHostToDevice, st));
      if (c) PSHT_CUDA_TRY(cudaMemcpyAsync(da + na, c, na, cudaMemcpyHostToDevice, st));
      exec_synthesis(p, da, c ? da + na : nullptr, p.d_io_f, st);
      PSHT_CUDA_TRY(cudaMemcpyAsync(f, p.d_io_f, (size_t)p.npts * cb, cudaMemcpyDeviceToHost, st));
    }
    PSHT_CUDA_TRY(cudaStreamSynchronize(st));
  });
}

int psht_plan_adjoint_host(psht_plan* plan, const void* f, void* g, void* c, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g && f, PSHT_EINVAL, "plan, f and g must not be NULL");
    Plan& p = *plan->p;
    cudaStream_t st = (cudaStream_t)stream;
    ensure_io(p);
    const size_t cb = p.prec == 64 ? 16 : 8, na = (size_t)p.nalm * cb;
    char* da = (char*)p.d_io_a;
    if (!p.chunk_m.empty() && !p.patch) {
      adjoint_host_chunked(p, f, g, c, st);
    } else {
      PSHT_CUDA_TRY(cudaMemcpyAsync(p.d_io_f, f, (size_t)p.npts * cb, cudaMemcpyHostToDevice, st));
      exec_adjoint(p, p.d_io_f, da, c ? da + na : nullptr, st);
      PSHT_CUDA_TRY(cudaMemcpyAsync(g, da, na, cudaMemcpyDeviceToHost, st));
      if (c) PSHT_CUDA_TRY(cudaMemcpyAsync(c, da + na, na, cudaMemcpyDeviceToHost, st));
    }
    PSHT_CUDA_TRY(cudaStreamSynchronize(st));
  });
}

int psht_plan_destroy(psht_plan* plan) {
  if (!plan) return PSHT_OK;
  destroy(plan->p);
  delete plan;
  return PSHT_OK;
}

int psht_plan_rings(const psht_plan* plan, double* theta_j, double* w_j, int32_t* Mj) {
  return guarded([&] {
    PSHT_REQUIRE(plan, PSHT_EINVAL, "plan must not be NULL");
    const Plan& p = *plan->p;
    for (int j = 0; j < p.nring; ++j) {
      if (theta_j) theta_j[j] = p.theta_j[j];
      if (w_j) w_j[j] = p.w_j[j];
      if (Mj) Mj[j] = p.Mj[j];
    }
  });
}

int psht_plan_ring_coeffs(psht_plan* plan, const void* g, const void* c, void* F, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && g && F, PSHT_EINVAL, "plan, g and F must not be NULL");
    Plan& p = *plan->p;
    if (p.patch) {  // the rings live in the plan's frame
      const size_t na = (size_t)p.nalm * (p.prec == 64 ? 16 : 8);
      char* ra = (char*)p.d_ra;
      rotator_apply(*p.rot, p.euler[0], p.euler[1], p.euler[2], g, c, ra, c ? ra + na : nullptr,
                    (cudaStream_t)stream);
      g = ra;
      c = c ? ra + na : nullptr;
    }
    launch_rec_synthesis(*plan->p, g, c, (cudaStream_t)stream);
    launch_ring_coeffs_export(*plan->p, F, (cudaStream_t)stream);
  });
}

int psht_plan_status(psht_plan* plan, int* status, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(plan && status, PSHT_EINVAL, "plan and status must not be NULL");
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    PSHT_CUDA_TRY(cudaMemcpyAsync(&h, plan->p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSHT_CUDA_TRY(cudaMemsetAsync(plan->p->d_status, 0, sizeof(int), st));
    PSHT_CUDA_TRY(cudaStreamSynchronize(st));
    *status = h;
  });
}

int psht_plan_profile(psht_plan* plan, int enable) {
  return guarded([&] {
    PSHT_REQUIRE(plan, PSHT_EINVAL, "plan must not be NULL");
    plan->p->profile = enable != 0;
  });
}

int psht_plan_stage_times(psht_plan* plan, double* ms, int64_t* calls) {
  return guarded([&] {
    PSHT_REQUIRE(plan, PSHT_EINVAL, "plan must not be NULL");
    Plan& p = *plan->p;
    double acc[PSHT_NSTAGES] = {0};
    int64_t cnt[PSHT_NSTAGES] = {0};
    for (auto& r : p.recs) {
      PSHT_CUDA_TRY(cudaEventSynchronize(r.b));
      float t = 0.f;
      PSHT_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
      acc[r.stage] += t;
      cnt[r.stage] += 1;
      p.evpool.push_back(r.a);
      p.evpool.push_back(r.b);
    }
    p.recs.clear();
    for (int i = 0; i < PSHT_NSTAGES; ++i) {
      if (ms) ms[i] = acc[i];
      if (calls) calls[i] = cnt[i];
    }
  });
}

int psht_synthesis(const void* g, const void* c, int spin, int lmax, const double* theta, const double* phi,
                   int64_t npts, double eps, void* f, void* stream) {
  return guarded([&] {
    Plan* p = create(spin, lmax, theta, phi, npts, eps, PSHT_AUTO, nullptr, (cudaStream_t)stream);
    try {
      PSHT_REQUIRE(g && (f || npts == 0), PSHT_EINVAL, "g and f must not be NULL");
      run_synthesis(*p, g, c, f, (cudaStream_t)stream);
      PSHT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    } catch (...) {
      destroy(p);
      throw;
    }
    destroy(p);
  });
}

int psht_adjoint_synthesis(const void* f, int spin, int lmax, const double* theta, const double* phi, int64_t npts,
                           double eps, void* g, void* c, void* stream) {
  return guarded([&] {
    Plan* p = create(spin, lmax, theta, phi, npts, eps, PSHT_AUTO, nullptr, (cudaStream_t)stream);
    try {
      PSHT_REQUIRE(g && (f || npts == 0), PSHT_EINVAL, "f and g must not be NULL");
      run_adjoint(*p, f, g, c, (cudaStream_t)stream);
      PSHT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    } catch (...) {
      destroy(p);
      throw;
    }
    destroy(p);
  });
}

size_t psht_estimate_bytes(int spin, int lmax, double theta_star, int64_t npts, double eps, uint32_t flags) {
  try {
    Plan p;
    p.spin = spin;
    p.lmax = lmax;
    p.eps = eps;
    const uint32_t pf = flags & 3u;
    p.prec = (pf == PSHT_FP64) ? 64 : (pf == PSHT_FP32) ? 32 : (eps >= 1e-5 ? 32 : 64);
    p.npts = npts;
    p.force_full = (flags & PSHT_FULL_SKY) ? 1 : 0;
    p.patch = (flags & PSHT_PATCH_FRAME) ? 1 : 0;
    p.pole = 1;
    layout(p, theta_star);
    return planned_bytes(p);
  } catch (...) {
    return 0;
  }
}

int psht_plan_estimate_points(int spin, int lmax, const double* theta, const double* phi, int64_t npts, double eps,
                              uint32_t flags, void* stream, size_t* bytes) {
  return guarded([&] {
    PSHT_REQUIRE(bytes != nullptr, PSHT_EINVAL, "bytes must not be NULL");
    PSHT_REQUIRE(npts >= 0 && npts < ((int64_t)1 << 31), PSHT_EINVAL, "npts must lie in [0, 2^31)");
    PSHT_REQUIRE(npts == 0 || (theta && phi), PSHT_EINVAL, "theta and phi must be device pointers");
    PSHT_REQUIRE(eps >= 1e-14 && eps <= 1e-1, PSHT_EINVAL, "eps must lie in [1e-14, 1e-1]");
    PSHT_REQUIRE(spin >= 0 && lmax >= spin && lmax <= 65535, PSHT_EINVAL, "invalid spin or lmax");
    double red[3];
    reduce_points(theta, phi, npts, red, (cudaStream_t)stream);
    PSHT_REQUIRE(red[2] == 0.0, PSHT_EINVAL, "theta outside [0, pi], NaN, or non-finite phi in the points");
    if ((flags & PSHT_PATCH_FRAME) && npts > 0) {  // theta* in the patch-centred frame
      double eul[3], ts = 0.0;
      patch_rotation_device(theta, phi, npts, eul, &ts, (cudaStream_t)stream);
      red[0] = ts;
      red[1] = M_PI;
    }
    Plan p;
    p.spin = spin;
    p.lmax = lmax;
    p.eps = eps;
    const uint32_t pf = flags & 3u;
    p.prec = (pf == PSHT_FP64) ? 64 : (pf == PSHT_FP32) ? 32 : (eps >= 1e-5 ? 32 : 64);
    p.npts = npts;
    p.force_full = (flags & PSHT_FULL_SKY) ? 1 : 0;
    p.patch = (flags & PSHT_PATCH_FRAME) ? 1 : 0;
    p.pole = (red[0] <= red[1]) ? 1 : -1;
    layout(p, p.pole > 0 ? red[0] : red[1]);
    *bytes = planned_bytes(p);
  });
}

int psht_predict_error(int spin, int lmax, double theta_star, double eps, const psht_options* opt, const double* cl,
                       const double* beta, int n, double* rel_rms, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(spin >= 0 && lmax >= spin && lmax <= 65535, PSHT_EINVAL, "invalid spin or lmax");
    PSHT_REQUIRE(eps >= 1e-14 && eps <= 1e-1, PSHT_EINVAL, "eps must lie in [1e-14, 1e-1]");
    PSHT_REQUIRE(theta_star > 0.0 && theta_star <= M_PI, PSHT_EINVAL, "theta_star must lie in (0, pi]");
    PSHT_REQUIRE(cl && beta && rel_rms && n >= 0, PSHT_EINVAL, "cl, beta and rel_rms must not be NULL");
    for (int l = 0; l <= lmax; ++l) PSHT_REQUIRE(cl[l] >= 0.0, PSHT_EINVAL, "C_l must be >= 0");
    if (n == 0) return;
    Plan p;
    p.spin = spin;
    p.lmax = lmax;
    p.eps = eps;
    p.prec = 64;
    p.pole = 1;
    apply_options(p, opt);
    layout(p, theta_star);
    predict_error_device(p, make_seeds(lmax, spin), cl, beta, n, rel_rms, (cudaStream_t)stream);
  });
}

static int rot_prec(uint32_t flags) { return (flags & 3u) == PSHT_FP32 ? 32 : 64; }

int psht_rotator_create(int lmax, uint32_t flags, void* stream, psht_rotator** out) {
  return guarded([&] {
    PSHT_REQUIRE(out, PSHT_EINVAL, "out must not be NULL");
    *out = reinterpret_cast<psht_rotator*>(rotator_create(lmax, rot_prec(flags), (cudaStream_t)stream));
  });
}

int psht_rotator_apply(psht_rotator* rot, double alpha, double beta, double gamma, const void* g, const void* c,
                       void* g_out, void* c_out, void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(rot, PSHT_EINVAL, "rotator must not be NULL");
    rotator_apply(*reinterpret_cast<Rotator*>(rot), alpha, beta, gamma, g, c, g_out, c_out, (cudaStream_t)stream);
  });
}

int psht_rotator_destroy(psht_rotator* rot) {
  rotator_destroy(reinterpret_cast<Rotator*>(rot));
  return PSHT_OK;
}

size_t psht_rotator_bytes(int lmax, uint32_t flags) {
  return lmax < 0 ? 0 : rotator_bytes(lmax, rot_prec(flags));
}

int psht_rotate_alm(int lmax, double alpha, double beta, double gamma, const void* g, const void* c, void* g_out,
                    void* c_out, uint32_t flags, void* stream) {
  return guarded([&] {
    cudaStream_t st = (cudaStream_t)stream;
    Rotator* r = rotator_create(lmax, rot_prec(flags), st);
    try {
      rotator_apply(*r, alpha, beta, gamma, g, c, g_out, c_out, st);
      PSHT_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
      rotator_destroy(r);
      throw;
    }
    rotator_destroy(r);
  });
}

int psht_rotate_points(double alpha, double beta, double gamma, const double* theta, const double* phi, int64_t npts,
                       double* theta_out, double* phi_out, double* psi_out, void* stream) {
  return guarded([&] {
    rotate_points_device(alpha, beta, gamma, theta, phi, npts, theta_out, phi_out, psi_out, (cudaStream_t)stream);
  });
}

int psht_patch_rotation(const double* theta, const double* phi, int64_t npts, double* euler, double* theta_star,
                        void* stream) {
  return guarded([&] {
    PSHT_REQUIRE(npts > 0 && theta && phi && euler, PSHT_EINVAL, "patch rotation: need at least one point");
    double red[3];
    reduce_points(theta, phi, npts, red, (cudaStream_t)stream);
    PSHT_REQUIRE(red[2] == 0.0, PSHT_EINVAL, "theta outside [0, pi], NaN, or non-finite phi in the points");
    patch_rotation_device(theta, phi, npts, euler, theta_star, (cudaStream_t)stream);
  });
}

const char* psht_last_error(void) { return g_err.c_str(); }

const char* psht_version(void) { return "psht 0.1 (sm_103a)"; }

}  // extern "C"

extern "C" {

int psht_ring_synthesis_noalloc(int spin, int lmax, const double* theta, int nring, const void* g, const void* c,
                                void* F, void* stream) {
  return guarded([&] { ring_synthesis_noalloc(spin, lmax, theta, nring, g, c, F, (cudaStream_t)stream); });
}

size_t psht_noalloc_scratch_bytes(void) { return noalloc_scratch_bytes(); }

}  // extern "C"
