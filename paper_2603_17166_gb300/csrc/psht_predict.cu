// Error predictor of the partial-sky route (Sec. II.E), psht_predict_error.
//
// For a statistically isotropic field with spectrum C_l the power along a great circle through the
// pole is c_m = sum_l C_l (2l+1)/2 |d^l_{m,-s}(pi/2)|^2 (eq. cm for spin 0, eq. cms for spin s, with
// C_l = C^E_l + C^B_l), and the route's error at angle beta from the pole is
//   sigma^2(beta) = (1/2pi) sum_m c_m sigma_m^2(beta)                                      (eq. st)
// where sigma_m^2 is the error on the single wave e^{i m theta} after weighting by w and band
// limiting on the plan's ring samples (eq. s2m).  On the doubled circle the 2L samples sit at
// Theta_k = k pi/L, k = 0 .. 2L-1 (theta_k = Theta_k theta_max/pi, negative past the pole), and the
// band limit |n| <= L-1 reconstructs with the Dirichlet kernel
//   D(delta) = (1/2L) sum_{|n| <= L-1} e^{i n delta} = sin((2L-1) delta/2) / (2L sin(delta/2)).
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "psht_common.cuh"

namespace psht {

namespace {

// c_{+m} (column d_{m,-s}) and c_{-m} (column d_{m,s}) for one order m per thread: the normalised
// columns e = N_l d^l_{m,-+s}(pi/2) follow e_{l+1} = (+-B_l) e_l - C_l e_{l-1} (x = cos(pi/2) = 0),
// started from Wigner's closed form at l0 = max(m, s); at pi/2 they neither underflow nor grow.
// (2l+1)/2 |d|^2 = 2 pi e^2.
__global__ void k_cm(int lmax, int s, const MSeed* __restrict__ seeds, const double* __restrict__ cl,
                     double* __restrict__ cp, double* __restrict__ cmn) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > lmax) return;
  const MSeed sd = seeds[m];
  const double m2 = (double)m * m, s2 = (double)s * s;
  // log2 of the seed magnitude at half-angle pi/4: cos = sin = 2^-1/2
  const double lg = sd.lbin - 0.5 * (double)(sd.p1 + sd.q1);
  double e1 = sd.sign1 * exp2(lg), e2 = sd.sign2 * exp2(lg);
  double p1 = 0.0, p2 = 0.0, q1 = 0.0, q2 = 0.0;  // e at l-1
  for (int l = sd.l0; l <= lmax; ++l) {
    q1 += cl[l] * e1 * e1;
    q2 += cl[l] * e2 * e2;
    if (l == lmax) break;
    const double lp1 = l + 1.0;
    const double a = lp1 * (2.0 * l + 1.0) / sqrt((lp1 * lp1 - m2) * (lp1 * lp1 - s2));
    const double A = sqrt((2.0 * l + 3.0) / (2.0 * l + 1.0)) * a;
    const double B = (l == 0) ? 0.0 : A * (double)m * (double)s / ((double)l * lp1);
    double C = 0.0;
    if (l > sd.l0) {
      const double c = sqrt(((double)l * l - m2) * ((double)l * l - s2)) / ((double)l * (2.0 * l + 1.0));
      C = sqrt((2.0 * l + 3.0) / (2.0 * l - 1.0)) * a * c;
    }
    const double n1 = B * e1 - C * p1, n2 = -B * e2 - C * p2;
    p1 = e1;
    p2 = e2;
    e1 = n1;
    e2 = n2;
  }
  cp[m] = 2.0 * M_PI * q1;
  cmn[m] = 2.0 * M_PI * q2;
}

// One block per prediction angle beta_i: sum over the waves m in [-lmax, lmax] of c_m sigma_m^2.
// Per block the Dirichlet weights of the doubled-circle samples are folded onto the rings j = 0..L:
//   S_m = sum_j u_j cos(m beta_j) + i v_j sin(m beta_j),  u, v = w_j (D(Theta_i - Theta_j) +- D(Theta_i + Theta_j))
// (the mirrored sample of ring j, 0 < j < L, sits at -Theta_j with the same weight).
__global__ void k_sigma(int lmax, int L, double theta_max, const double* __restrict__ wj,
                        const double* __restrict__ beta, const double* __restrict__ cp,
                        const double* __restrict__ cmn, double* __restrict__ out) {
  extern __shared__ double sm[];
  double* u = sm;              // [L + 1]
  double* v = sm + (L + 1);    // [L + 1]
  __shared__ double red[32];
  const double bi = beta[blockIdx.x];
  const double Ti = bi * (M_PI / theta_max);
  const double h = M_PI / L;
  auto dir = [&](double d) {
    const double sh = sin(0.5 * d);
    if (fabs(sh) < 1e-300) return (2.0 * L - 1.0) / (2.0 * L);
    return sin((L - 0.5) * d) / (2.0 * L * sh);
  };
  for (int j = threadIdx.x; j <= L; j += blockDim.x) {
    const double a = dir(Ti - j * h);
    const double b = (j >= 1 && j <= L - 1) ? dir(Ti + j * h) : 0.0;
    u[j] = wj[j] * (a + b);
    v[j] = wj[j] * (a - b);
  }
  __syncthreads();
  const double dlt = theta_max / L;  // beta_j = j dlt
  double acc = 0.0;
  for (int mm = threadIdx.x; mm <= 2 * lmax; mm += blockDim.x) {
    const int m = mm - lmax;
    const double c = m >= 0 ? cp[m] : cmn[-m];
    if (c == 0.0) continue;
    double zs, zc;
    sincos(m * dlt, &zs, &zc);
    double pr = 1.0, pi = 0.0, sr = 0.0, si = 0.0;  // (pr, pi) = e^{i m j dlt}
    for (int j = 0; j <= L; ++j) {
      sr += u[j] * pr;
      si += v[j] * pi;
      const double t = pr * zc - pi * zs;
      pi = pr * zs + pi * zc;
      pr = t;
    }
    double er, ei;
    sincos(m * bi, &ei, &er);
    const double dr = sr - er, di = si - ei;
    acc += c * (dr * dr + di * di);
  }
  // block reduction
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
  }
}

}  // namespace

void predict_error_device(const Plan& p, const std::vector<MSeed>& seeds, const double* cl, const double* beta, int n,
                          double* rel_rms, cudaStream_t st) {
  const int lmax = p.lmax;
  const int L = p.L;
  std::vector<double> w(L + 1, 0.0);
  for (int j = 0; j <= L && j < p.nring; ++j) w[j] = p.w_j[j];
  double *d_cl = nullptr, *d_cp = nullptr, *d_cm = nullptr, *d_w = nullptr, *d_beta = nullptr, *d_out = nullptr;
  MSeed* d_seed = nullptr;
  auto cleanup = [&] {
    for (void* q : {(void*)d_cl, (void*)d_cp, (void*)d_cm, (void*)d_w, (void*)d_beta, (void*)d_out, (void*)d_seed})
      if (q) cudaFreeAsync(q, st);
  };
  try {
    PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_cl, sizeof(double) * (lmax + 1), st));
    PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_cp, sizeof(double) * (lmax + 1), st));
    PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_cm, sizeof(double) * (lmax + 1), st));
    PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_w, sizeof(double) * (L + 1), st));
    PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_beta, sizeof(double) * n, st));
    PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_out, sizeof(double) * n, st));
    PSHT_CUDA_TRY(cudaMallocAsync((void**)&d_seed, sizeof(MSeed) * (lmax + 1), st));
    PSHT_CUDA_TRY(cudaMemcpyAsync(d_cl, cl, sizeof(double) * (lmax + 1), cudaMemcpyHostToDevice, st));
    PSHT_CUDA_TRY(cudaMemcpyAsync(d_w, w.data(), sizeof(double) * (L + 1), cudaMemcpyHostToDevice, st));
    PSHT_CUDA_TRY(cudaMemcpyAsync(d_beta, beta, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    PSHT_CUDA_TRY(cudaMemcpyAsync(d_seed, seeds.data(), sizeof(MSeed) * (lmax + 1), cudaMemcpyHostToDevice, st));
    k_cm<<<(lmax + 128) / 128, 128, 0, st>>>(lmax, p.spin, d_seed, d_cl, d_cp, d_cm);
    PSHT_CUDA_TRY(cudaGetLastError());
    const size_t smem = sizeof(double) * 2 * (L + 1);
    allow_dynamic_smem((const void*)k_sigma, smem);
    k_sigma<<<n, 256, smem, st>>>(lmax, L, p.theta_max, d_w, d_beta, d_cp, d_cm, d_out);
    PSHT_CUDA_TRY(cudaGetLastError());
    std::vector<double> cp(lmax + 1), cm(lmax + 1);
    PSHT_CUDA_TRY(cudaMemcpyAsync(rel_rms, d_out, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    PSHT_CUDA_TRY(cudaMemcpyAsync(cp.data(), d_cp, sizeof(double) * (lmax + 1), cudaMemcpyDeviceToHost, st));
    PSHT_CUDA_TRY(cudaMemcpyAsync(cm.data(), d_cm, sizeof(double) * (lmax + 1), cudaMemcpyDeviceToHost, st));
    PSHT_CUDA_TRY(cudaStreamSynchronize(st));
    cleanup();
    double var = cp[0];
    for (int m = 1; m <= lmax; ++m) var += cp[m] + cm[m];
    for (int i = 0; i < n; ++i) rel_rms[i] = var > 0.0 ? sqrt(rel_rms[i] / var) : 0.0;
  } catch (...) {
    cleanup();
    throw;
  }
}

}  // namespace psht
