// Allocation-free ring synthesis (psht_ring_synthesis_noalloc in include/psht.h).
//
// Some callers cannot allocate device memory: their device memory is fully owned by another
// allocator (a framework's caching pool, a memory-capped service), or they must not call
// cudaMalloc/cudaFree, which can synchronise the whole device, in the middle of their own work.
// This entry point serves them: it computes the same ring Fourier coefficients as
// psht_plan_ring_coeffs without a plan, keeping every intermediate (recurrence table, ring data,
// seeds) in one file-scope device array of fixed size.  It is FP64 and limited to lmax <= 511 and
// at most 4096 rings.
//
// The array is shared by all calls on a device and keeps the last call's contents; each call
// rewrites everything it reads, so nothing has to start at zero.  Calls whose work overlaps on
// the GPU (different streams, or different host threads) race on the array and must be ordered
// by the caller.  The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (with that device current); make that first call before any stream
// capture.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "psht_common.cuh"

namespace psht {
namespace {

constexpr int kNaLmax = PSHT_NOALLOC_MAX_LMAX;
constexpr int kNaRings = PSHT_NOALLOC_MAX_RINGS;
constexpr int64_t kNaNalm = (int64_t)(kNaLmax + 1) * (kNaLmax + 2) / 2;
constexpr size_t kTabBytes = (size_t)4 * kNaNalm * sizeof(double);  // A, D, B, C per (l, m)
struct NaRing {                                                  // one ring, evaluated at b <= pi/2
  double omx, l2c, l2s;
  int refl;
  int pad;
};
struct NaSeed {
  double lbin;
  int l0, p1, q1, sign1, sign2, pad;
};
constexpr size_t kRingOff = (kTabBytes + 255) / 256 * 256;
constexpr size_t kSeedOff = kRingOff + ((size_t)kNaRings * sizeof(NaRing) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kSeedOff + (size_t)(kNaLmax + 1) * sizeof(NaSeed);

// the scratch array: every GPU that loads the library holds it until the process exits
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__device__ __forceinline__ int64_t na_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// per-ring data from the caller's colatitudes; rings past the equator are evaluated by the
// reflection d^l_{m,-s}(pi - b) = (-1)^(l+m) d^l_{m,s}(b)
__global__ void k_na_rings(const double* __restrict__ theta, int nring, NaRing* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nring) return;
  const double t = theta[j];
  const int refl = t > 0.5 * M_PI;
  const double b = refl ? M_PI - t : t;
  const double sb = sin(0.5 * b), cb = cos(0.5 * b);
  NaRing r;
  r.omx = 2.0 * sb * sb;
  r.l2c = cb > 0 ? log2(cb) : -INFINITY;
  r.l2s = sb > 0 ? log2(sb) : -INFINITY;
  r.refl = refl;
  r.pad = 0;
  out[j] = r;
}

// per order m: Wigner's closed-form seed at l0 = max(m, s) as log2 magnitude and signs, and the
// recurrence coefficients of every l (FP64)
__global__ void k_na_setup(int lmax, int s, double* __restrict__ tab, int64_t ts, NaSeed* __restrict__ seeds) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > lmax) return;
  NaSeed d;
  d.l0 = max(m, s);
  if (m >= s) {
    d.p1 = m - s;
    d.q1 = m + s;
    d.sign1 = d.sign2 = ((m + s) & 1) ? -1 : 1;
  } else {
    d.p1 = s - m;
    d.q1 = s + m;
    d.sign1 = ((s + m) & 1) ? -1 : 1;
    d.sign2 = 1;
  }
  const double l0 = d.l0;
  d.lbin = 0.5 * (lgamma(2.0 * l0 + 1.0) - lgamma(d.p1 + 1.0) - lgamma(d.q1 + 1.0)) / log(2.0) +
           0.5 * log2((2.0 * l0 + 1.0) / (4.0 * M_PI));
  d.pad = 0;
  seeds[m] = d;
  const int64_t base = na_base(lmax, m);
  const double m2 = (double)m * m, s2 = (double)s * s;
  for (int l = m; l <= lmax; ++l) {
    double A = 0, B = 0, C = 0;
    if (l >= d.l0 && l < lmax) {
      const double lp1 = l + 1.0;
      const double a = lp1 * (2.0 * l + 1.0) / sqrt((lp1 * lp1 - m2) * (lp1 * lp1 - s2));
      A = sqrt((2.0 * l + 3.0) / (2.0 * l + 1.0)) * a;
      B = (l == 0) ? 0.0 : A * (double)m * (double)s / ((double)l * lp1);
      if (l > d.l0) {
        const double c = sqrt(((double)l * l - m2) * ((double)l * l - s2)) / ((double)l * (2.0 * l + 1.0));
        C = sqrt((2.0 * l + 3.0) / (2.0 * l - 1.0)) * a * c;
      }
    }
    tab[base + l] = A;
    tab[ts + base + l] = (A - 1.0) - C;
    tab[2 * ts + base + l] = B;
    tab[3 * ts + base + l] = C;
  }
}

__device__ __forceinline__ void na_seed(double lg, int sign, double& e, int& k) {
  // value held as e 2^(-500 k); contributions below 2^-100 are dropped while k > 0
  if (!(lg > -1.0e30)) {
    e = 0.0;
    k = 1;
    return;
  }
  k = 0;
  if (lg < -100.0) {
    k = (int)ceil((-100.0 - lg) / 500.0);
    lg += 500.0 * k;
  }
  e = sign * exp2(lg);
}

__device__ __forceinline__ void na_step(double t, double C, double& e, double& d, int& k) {
  d = fma(t, e, C * d);
  e = e + d;
  if (k > 0 && fabs(e) >= 0x1p400) {
    e *= 0x1p-500;
    d *= 0x1p-500;
    --k;
  }
}

// one thread per (ring, m >= 0): F[j][m + lmax] and F[j][-m + lmax], the scaled Reinsch recurrence
// of both Wigner columns (same mathematics as the planned path's synthesis recursion)
__global__ void k_na_rings_synth(int lmax, int s, int nring, const NaRing* __restrict__ rings,
                                 const NaSeed* __restrict__ seeds, const double* __restrict__ tab, int64_t ts,
                                 const double2* __restrict__ g, const double2* __restrict__ c,
                                 double2* __restrict__ F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (j >= nring || m > lmax) return;
  const NaRing rg = rings[j];
  const NaSeed sd = seeds[m];
  double e1, e2, d1, d2;
  int k1, k2;
  na_seed(sd.lbin + (sd.p1 > 0 ? sd.p1 * rg.l2c : 0.0) + (sd.q1 > 0 ? sd.q1 * rg.l2s : 0.0), sd.sign1, e1, k1);
  na_seed(sd.lbin + (sd.q1 > 0 ? sd.q1 * rg.l2c : 0.0) + (sd.p1 > 0 ? sd.p1 * rg.l2s : 0.0), sd.sign2, e2, k2);
  d1 = e1;
  d2 = e2;
  const int64_t base = na_base(lmax, m);
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int l = sd.l0; l <= lmax; ++l) {
    double2 gv = g[base + l];
    double2 cv = c ? c[base + l] : make_double2(0.0, 0.0);
    if (m == 0) {
      gv.y = 0.0;
      cv.y = 0.0;
    }
    // u = g + i c pairs with d_{m,-s}(theta), v = g* + i c* with d_{m,s}(theta); a reflected ring
    // swaps the columns and signs the coefficients by (-1)^(l+m)
    double ur = gv.x - cv.y, ui = gv.y + cv.x, vr = gv.x + cv.y, vi = cv.x - gv.y;
    double P0 = ur, P1 = ui, Q0 = vr, Q1 = vi;
    if (rg.refl) {
      const double sg = ((l + m) & 1) ? -1.0 : 1.0;
      P0 = sg * vr;
      P1 = sg * vi;
      Q0 = sg * ur;
      Q1 = sg * ui;
    }
    const double o1 = k1 == 0 ? e1 : 0.0, o2 = k2 == 0 ? e2 : 0.0;
    a0 = fma(P0, o1, a0);
    a1 = fma(P1, o1, a1);
    a2 = fma(Q0, o2, a2);
    a3 = fma(Q1, o2, a3);
    if (l < lmax) {
      const double t = fma(-tab[base + l], rg.omx, tab[ts + base + l]);
      const double B = tab[2 * ts + base + l], C = tab[3 * ts + base + l];
      na_step(t + B, C, e1, d1, k1);
      na_step(t - B, C, e2, d2, k2);
    }
  }
  const double sgn_s = (s & 1) ? 1.0 : -1.0;  // -(-1)^s
  const double2 fpos = rg.refl ? make_double2(-a2, -a3) : make_double2(-a0, -a1);
  const double2 fneg = rg.refl ? make_double2(sgn_s * a0, sgn_s * a1) : make_double2(sgn_s * a2, sgn_s * a3);
  const int64_t row = (int64_t)j * (2 * lmax + 1);
  F[row + lmax + m] = fpos;
  if (m > 0) F[row + lmax - m] = fneg;
}

// device address of the scratch array, looked up once per device
std::mutex g_na_mutex;
void* g_na_ptr[64] = {nullptr};

void* noalloc_scratch() {
  int dev = 0;
  PSHT_CUDA_TRY(cudaGetDevice(&dev));
  PSHT_REQUIRE(dev >= 0 && dev < 64, PSHT_ENOTSUP, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* ptr = nullptr;
    PSHT_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_na_ptr[dev] = ptr;
  }
  return g_na_ptr[dev];
}

}  // namespace

void ring_synthesis_noalloc(int spin, int lmax, const double* theta, int nring, const void* g, const void* c, void* F,
                            cudaStream_t st) {
  PSHT_REQUIRE(spin >= 0 && lmax >= spin, PSHT_EINVAL, "need 0 <= spin <= lmax");
  PSHT_REQUIRE(lmax <= kNaLmax, PSHT_EINVAL,
               "lmax above " + std::to_string(kNaLmax) + ", the fixed scratch size of the allocation-free call");
  PSHT_REQUIRE(nring >= 0 && nring <= kNaRings, PSHT_EINVAL,
               "nring above " + std::to_string(kNaRings) + ", the fixed scratch size of the allocation-free call");
  PSHT_REQUIRE(nring == 0 || (theta && g && F), PSHT_EINVAL, "theta, g and F must be device pointers");
  if (nring == 0) return;
  unsigned char* base = (unsigned char*)noalloc_scratch();
  const int64_t ts = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  double* tab = (double*)base;
  NaRing* rings = (NaRing*)(base + kRingOff);
  NaSeed* seeds = (NaSeed*)(base + kSeedOff);
  k_na_rings<<<(nring + 127) / 128, 128, 0, st>>>(theta, nring, rings);
  k_na_setup<<<(lmax + 1 + 127) / 128, 128, 0, st>>>(lmax, spin, tab, ts, seeds);
  const dim3 grid((nring + 127) / 128, lmax + 1);
  k_na_rings_synth<<<grid, 128, 0, st>>>(lmax, spin, nring, rings, seeds, tab, ts, (const double2*)g,
                                         (const double2*)c, (double2*)F);
  PSHT_CUDA_TRY(cudaGetLastError());
}

size_t noalloc_scratch_bytes() { return kScratchBytes; }

}  // namespace psht
