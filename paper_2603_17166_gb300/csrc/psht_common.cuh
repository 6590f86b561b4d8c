// Device helpers shared by the psht kernels: complex arithmetic, small DFTs and an in-place
// mixed-radix FFT held in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "psht_internal.h"

namespace psht {

template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using V = double2;
};
template <>
struct Cx<float> {
  using V = float2;
};

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a conj(b)
template <typename V, typename S>
__device__ __forceinline__ V cscale(V a, S s) { return mk(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V>
__device__ __forceinline__ V rot90(V a) { return INV ? mk(-a.y, a.x) : mk(a.y, -a.x); }

// ---------------------------------------------------------------------------------------------
// small DFTs y_q = sum_r x_r e^{-+2 pi i r q/R} (minus: forward, plus: INV), in place on v[R]
template <int R, bool INV, typename V>
struct Dft;

template <bool INV, typename V>
struct Dft<2, INV, V> {
  __device__ __forceinline__ static void run(V* v) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <bool INV, typename V>
struct Dft<4, INV, V> {
  __device__ __forceinline__ static void run(V* v) {
    V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    V t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};
template <bool INV, typename V>
struct Dft<8, INV, V> {
  __device__ __forceinline__ static void run(V* v) {
    using S = decltype(v[0].x);
    const S h = (S)0.707106781186547524400844362104849039;
    V e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV, V>::run(e);
    Dft<4, INV, V>::run(o);
    // twiddles e^{-+2 pi i k/8}, k = 0..3
    V o1 = INV ? mk(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y)) : mk(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    V o2 = rot90<INV>(o[2]);
    V o3 = INV ? mk(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y)) : mk(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};
template <bool INV, typename V>
struct Dft<3, INV, V> {
  __device__ __forceinline__ static void run(V* v) {
    using S = decltype(v[0].x);
    const S c = (S)0.866025403784438646763723170752936183;  // sin(2 pi/3)
    V t = cadd(v[1], v[2]);
    V u = mk(v[0].x - (S)0.5 * t.x, v[0].y - (S)0.5 * t.y);
    V d = rot90<INV>(cscale(csub(v[1], v[2]), c));
    v[0] = cadd(v[0], t);
    v[1] = cadd(u, d);
    v[2] = csub(u, d);
  }
};
// odd prime R: y_q = x_0 + sum_{n=1}^{(R-1)/2} [(x_n + x_{R-n}) cos(2 pi n q/R) -+ i (x_n - x_{R-n}) sin(2 pi n q/R)]
template <int R, bool INV, typename V>
struct DftOdd {
  __device__ __forceinline__ static void run(V* v, const double* cs, const double* sn) {
    using S = decltype(v[0].x);
    constexpr int H = (R - 1) / 2;
    V a[H], b[H];
#pragma unroll
    for (int n = 1; n <= H; ++n) {
      a[n - 1] = cadd(v[n], v[R - n]);
      b[n - 1] = csub(v[n], v[R - n]);
    }
    V y[R];
    V s0 = v[0];
#pragma unroll
    for (int n = 0; n < H; ++n) s0 = cadd(s0, a[n]);
    y[0] = s0;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      V re = v[0], im = mk((S)0, (S)0);
#pragma unroll
      for (int n = 1; n <= H; ++n) {
        const int idx = (n * q) % R;  // cos/sin of 2 pi idx/R, tables hold idx = 1..H, symmetric
        const int k = idx <= H ? idx : R - idx;
        const S cc = (S)cs[k - 1];
        const S ss = (S)(idx <= H ? sn[k - 1] : -sn[k - 1]);
        re = mk(re.x + cc * a[n - 1].x, re.y + cc * a[n - 1].y);
        im = mk(im.x + ss * b[n - 1].x, im.y + ss * b[n - 1].y);
      }
      // forward: y_q = re - i im,  y_{R-q} = re + i im ; inverse: signs swapped
      V mi = rot90<INV>(im);  // -i im (forward) / +i im (inverse)
      y[q] = cadd(re, mi);
      y[R - q] = csub(re, mi);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = y[q];
  }
};
__device__ __constant__ static const double kCos5[2] = {0.309016994374947424102293417182819059,
                                                        -0.809016994374947424102293417182819059};
__device__ __constant__ static const double kSin5[2] = {0.951056516295153572116439333379382143,
                                                        0.587785252292473129168705954639072769};
__device__ __constant__ static const double kCos7[3] = {0.623489801858733530525004884004239811,
                                                        -0.222520933956314404288902564496794759,
                                                        -0.900968867902419126236102319507445051};
__device__ __constant__ static const double kSin7[3] = {0.78183148246802980870844452667405775,
                                                        0.974927912181823607018131682993931217,
                                                        0.433883739117558120475768332848358755};
template <bool INV, typename V>
struct Dft<5, INV, V> {
  __device__ __forceinline__ static void run(V* v) { DftOdd<5, INV, V>::run(v, kCos5, kSin5); }
};
template <bool INV, typename V>
struct Dft<7, INV, V> {
  __device__ __forceinline__ static void run(V* v) { DftOdd<7, INV, V>::run(v, kCos7, kSin7); }
};

// ---------------------------------------------------------------------------------------------
// Shared-memory FFT buffer with one pad element after every 32: the butterflies of the late DIF
// (early DIT) stages read with power-of-two strides, which put a warp's lanes on a few banks
// (stride 8 or 16: 8- to 16-way conflicts); with the pad those strides cost at most two ways,
// while the stride-1 accesses of the early stages stay on whole 256-byte rows (a pad after
// every 16 measured more conflicts in total: it splits those rows).
template <typename V>
struct PadBuf {
  V* p;
  __device__ __forceinline__ V& operator[](int i) const { return p[i + (i >> 5)]; }
};
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 5) + 1; }

// Twiddle e^{-2 pi i t/N}.  FP64: a full table tw[t].  FP32: the product of two short tables,
// tw[t mod 64] e^{-2 pi i 64 floor(t/64)/N} = tw[t & 63] tw[64 + (t >> 6)] (64 + N/64 + 1 entries),
// which stay in L1 next to the shared-memory buffers (the full tables did not); one extra complex
// multiply, error ~1e-7.
template <typename V>
__device__ __forceinline__ V twiddle(const V* __restrict__ tw, int t);
template <>
__device__ __forceinline__ double2 twiddle<double2>(const double2* __restrict__ tw, int t) {
  return __ldg(&tw[t]);
}
template <>
__device__ __forceinline__ float2 twiddle<float2>(const float2* __restrict__ tw, int t) {
  const float2 a = __ldg(&tw[t & 63]), b = __ldg(&tw[64 + (t >> 6)]);
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// ---------------------------------------------------------------------------------------------
// In-place mixed-radix FFT of length N in shared memory, all threads of the block cooperate.
// DIF (Gentleman-Sande): natural-order input, output frequency k at position perm[k].
// DIT (transpose of DIF): input n placed at perm[n], natural-order output.
// tw[t] = e^{-2 pi i t/N}; INV uses conj twiddles (unnormalised inverse).
// Each butterfly reads and writes the same R positions, so one buffer and R registers suffice.
template <int R, bool INV, bool DIF, typename V, typename B>
__device__ __forceinline__ void fft_stage(B buf, int N, int Nc, const V* __restrict__ tw) {
  const int s = Nc / R;
  const int nb = N / R;
  const int tstride = N / Nc;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int blk = b / s, j = b - blk * s;
    const int base = blk * Nc + j;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = buf[base + r * s];
    if (!DIF) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const V w = twiddle<V>(tw, j * q * tstride);
        v[q] = INV ? cmulc(v[q], w) : cmul(v[q], w);
      }
    }
    Dft<R, INV, V>::run(v);
    if (DIF) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const V w = twiddle<V>(tw, j * q * tstride);
        v[q] = INV ? cmulc(v[q], w) : cmul(v[q], w);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) buf[base + r * s] = v[r];
  }
}

template <bool INV, bool DIF, typename V, typename B>
__device__ __forceinline__ void fft_stage_dispatch(int R, B buf, int N, int Nc, const V* tw) {
  switch (R) {
    case 8: fft_stage<8, INV, DIF, V>(buf, N, Nc, tw); break;
    case 4: fft_stage<4, INV, DIF, V>(buf, N, Nc, tw); break;
    case 2: fft_stage<2, INV, DIF, V>(buf, N, Nc, tw); break;
    case 3: fft_stage<3, INV, DIF, V>(buf, N, Nc, tw); break;
    case 5: fft_stage<5, INV, DIF, V>(buf, N, Nc, tw); break;
    case 7: fft_stage<7, INV, DIF, V>(buf, N, Nc, tw); break;
    default: break;
  }
}

// The caller syncs before the call; the function syncs after every stage.
template <bool INV, typename V, typename B>
__device__ void fft_dif(B buf, const FftDev& f, const V* tw) {
  int Nc = f.n;
  for (int st = 0; st < f.nst; ++st) {
    const int R = f.rad[st];
    fft_stage_dispatch<INV, true, V>(R, buf, f.n, Nc, tw);
    Nc /= R;
    __syncthreads();
  }
}
template <bool INV, typename V, typename B>
__device__ void fft_dit(B buf, const FftDev& f, const V* tw) {
  int Nc = 1;
  for (int st = f.nst - 1; st >= 0; --st) {
    const int R = f.rad[st];
    Nc *= R;
    fft_stage_dispatch<INV, false, V>(R, buf, f.n, Nc, tw);
    __syncthreads();
  }
}

// digit-reversed position of natural index k for the radix schedule of f (DIF output order)
__device__ __forceinline__ int fft_pos(const FftDev& f, int k) {
  int p = 0, s = f.n;
  for (int st = 0; st < f.nst; ++st) {
    const int R = f.rad[st];
    s /= R;
    const int q = k % R;
    k /= R;
    p += q * s;
  }
  return p;
}

// ---------------------------------------------------------------------------------------------
// mbarrier + bulk copy helpers (inline PTX): a single thread arms the barrier with the expected
// byte count and issues cp.async.bulk; consumers wait on the barrier's phase parity, for at most
// kSpinLimit polls, after which the caller records a status and leaves instead of hanging.
constexpr int kSpinLimit = 1 << 26;
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after kSpinLimit polls (the caller reports it and leaves)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// m of column index mi: 0 -> 0, 2m -> +m, 2m-1 -> -m
__device__ __forceinline__ int col_m(int mi) { return (mi == 0) ? 0 : ((mi & 1) ? -((mi + 1) >> 1) : (mi >> 1)); }
__device__ __forceinline__ int col_of(int m) { return m >= 0 ? 2 * m : -2 * m - 1; }

}  // namespace psht
