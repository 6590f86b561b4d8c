// Internal declarations of the psht library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/psht.h"

namespace psht {

// ---------------------------------------------------------------------------------------------
// error handling
void set_error(const std::string& msg);
struct Error {
  int code;
  std::string msg;
};
#define PSHT_CUDA_TRY(call)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::psht::Error{PSHT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};   \
  } while (0)
#define PSHT_REQUIRE(cond, code, msg)                  \
  do {                                                 \
    if (!(cond)) throw ::psht::Error{(code), (msg)};   \
  } while (0)

// ---------------------------------------------------------------------------------------------
// constants of the scaled recursion.  A value is held as y * 2^(-F k) with k >= 0; while k > 0 the
// true value is below 2^(R_EXP - F) and its contribution is dropped.  The rescale test runs every
// 4 steps of l, so values may pass 2^R_EXP by the growth of 4 steps (< 2^32) before rescaling.
template <typename T>
struct ScaleConst;
// ring slots per lane of the FP32 synthesis recursion (packed pairs: a multiple of 2).  One pair
// measured faster than two at lmax 4096, also with the plan-time start states (1.94 against
// 2.04 ms): the same issue rate, and items of 64 rings leave fewer idle slots and shorter stretches
// of partly dropped columns than items of 128.
constexpr int kSynRpt32 = 2;
template <>
struct ScaleConst<double> {
  static constexpr int F = 500;      // exponent step of one rescale
  static constexpr int R_EXP = 400;  // rescale when |y| >= 2^400; dropped region below 2^-100
};
// FP64 rings at least this far from the pole (degrees) take the three-term form of the recurrence
// when eps >= kThreeTermMinEps (its error there stays within a few 1e-13 at lmax 4096)
constexpr double kThreeTermDeg = 10.0;
constexpr double kThreeTermMinEps = 1e-11;

template <>
struct ScaleConst<float> {
  static constexpr int F = 80;
  static constexpr int R_EXP = 20;   // dropped region below 2^(20-80) = 2^-60
};

// ---------------------------------------------------------------------------------------------
// device-side tables
struct RingDev {    // ring j evaluated at b = min(theta_j, pi - theta_j), its distance from the nearer pole
  double omx;       // 1 - cos(b) = 2 sin^2(b/2)
  double l2c, l2s;  // log2 cos(b/2), log2 sin(b/2)  (-inf allowed)
  float ohi, olo;   // omx split into two floats (FP32 form)
};

struct MSeed {      // per order m, for the two recursions m' = -s (e1) and m' = +s (e2)
  double lbin;      // log2( N_{l0} sqrt(C(2 l0, p1)) )
  int l0;           // max(m, s)
  int p1, q1;       // e1 seed ~ cos^p1 sin^q1 of the half angle (e2 uses cos^q1 sin^p1)
  int sign1, sign2; // signs of the two seeds
};

struct RecItem {    // one CTA of the synthesis recursion: order m, rings [j0, j0 + nj)
  int m, j0, nj;
  int refl;         // 1: the rings lie at theta > pi/2 and are evaluated at pi - theta (reflection)
};

struct AdjItem {    // one warp of the FP32 adjoint recursion: order m, rings [j0, j0 + nj)
  int m, j0, nj;
  int refl;
  int nitems;       // items of order m (1: the item projects its own sums; else they meet in d_acc)
};

// One-warp recursion items (FP32 synthesis and adjoint, FP64 synthesis): where each item (a warp's
// rings of one order) starts.  Below the first l at which any of the item's Wigner columns reaches
// the working range the kernels would only step dropped columns and sum nothing; the plan steps
// those l once, with the kernels' arithmetic and rescaling, and keeps each ring slot's state there,
// so every call starts at that l.
struct RecStart {
  int* ls = nullptr;        // per item: first l of its first quad with a working column (> lmax: none)
  void* st = nullptr;       // per item x slot x lane: (e1, d1, e2, d2) at ls, scaled as the kernels scale
                            // (FP32 float4; FP64 four doubles, d = e_{l-1} in the three-term form)
  int* kk = nullptr;        // per item x slot x lane: scale counts k1 | k2 << 16
};

struct TileItem {   // one CTA of the gather/scatter: a tile and a slice of its sorted points
  int tr, tq;       // tile row/column index
  int p0, np;       // first sorted point, count
};

struct FftDev {     // radix schedule of one FFT length (at most 32 stages)
  int n, nst;
  int rad[32];
};

// ---------------------------------------------------------------------------------------------
struct Rotator;  // Wigner-D rotation of a_lm sets (psht_rotate.cu)

struct Plan {
  // parameters (names as in the paper)
  int spin = 0, lmax = 0, prec = 64;
  double eps = 0;
  int pole = 1, full = 0;
  int force_full = 0;  // PSHT_FULL_SKY
  int window = 0;      // PSHT_WINDOW_ES or PSHT_WINDOW_KB
  double kappa = 1.0;  // ring-count factor in Lmax
  int apo_cost = 0;    // PSHT_APO_COST: eps_apo minimising the recursion's step count
  // FP64 rings with 1 - cos(b) >= omx_tb (b the distance from the pole) take the three-term form of
  // the recurrence instead of Reinsch's (above 2: none)
  double omx_tb = 3.0;
  double theta_star = 0, eps_apo = 0, theta_max = 0, dTheta = 0, alpha = 0;
  int Lmax = 0, L = 0, nring = 0, M = 0, W = 0;
  double beta_es = 0;
  int nTheta = 0, nphi = 0, r_lo = 0, nrows = 0;
  int64_t npts = 0, nalm = 0;
  std::vector<double> theta_j, beta_j, w_j;
  std::vector<int> Mj;
  // layouts
  int ncols = 0;    // 2M+1 columns of the ring / row arrays, column mi(m) = 2m (m>=0), 2|m|-1 (m<0)
  int Lpad = 0;     // leading dimension of F (ring index fastest)
  int padq = 0;     // grid columns stored at q + padq, q in [-padq, nphi + padq)
  int gstride = 0;  // grid row stride (complex elements)
  int TR = 0, TQ = 0, ntr = 0, ntq = 0;
  // recursion launch shapes
  int syn_rpt = 1, syn_threads = 128, adj_rpt = 1, adj_threads = 128;
  int64_t pairs = 0, triples = 0;
  // device memory
  RingDev* d_ring = nullptr;
  MSeed* d_mseed = nullptr;
  int2* d_mrange = nullptr;     // active ring range [j_lo, j_hi) per m: part 0 (theta <= pi/2), then part 1
  int has_refl = 0;             // any ring at theta > pi/2 (part 1 non-empty)
  void* d_rtab = nullptr;       // recurrence table: one record per packed (l, m) (32 B FP64, 48 B FP32), padded by one chunk
  int64_t tstride = 0;          // records in the table (nalm + one chunk of zero records)
  int* d_status = nullptr;      // device error word (bounded waits that gave up), read by psht_plan_status
  RecItem* d_items = nullptr;
  int nitems = 0;
  // full-sky plans: rings j and nring - 1 - j lie at b and pi - b and share their Wigner columns;
  // orders whose reflected active rings are exactly the mirrors of their direct ones run as pairs
  RecItem* d_mitems = nullptr;  // synthesis items of mirror pairs (direct rings j of the pairs)
  int nmitems = 0;
  AdjItem* d_maitems = nullptr; // FP32 adjoint items of mirror pairs
  int nmaitems = 0;
  int* d_mmode = nullptr;       // per m: 1 if the order runs as mirror pairs (FP64 block adjoint), else null
  AdjItem* d_aitems = nullptr;  // adjoint as one warp per item (adj_threads == 32)
  int naitems = 0;
  int2* d_aspan = nullptr;      // per m: first adjoint item, item count
  void* d_acc = nullptr;        // FP32 adjoint: float4 [nalm], the sums of orders with several items
  int* d_cnt = nullptr;         // FP32 adjoint: per m, items of that order finished in the current call
  // start states of the synthesis items, mirror items (both forms), FP32 adjoint items and FP32
  // mirror adjoint items
  RecStart s_items, s_mitems, s_aitems, s_maitems;
  // FP64 block adjoint: per launch (ring part x ring chunk) and order m, the CTA's first working l
  // (s_badj.ls[launch * (M + 1) + m]) and each active ring's state there (four doubles and the
  // scale counts at s_badj_off[launch * (M + 1) + m] + the ring's index in the chunk)
  RecStart s_badj;
  int64_t* s_badj_off = nullptr;
  int badj_nch = 0;  // ring chunks per part
  // batched execution (psht_plan_*_batch): ring coefficients and (FP32) accumulators of the sets
  // after the first of a group, allocated on the first batched call
  std::vector<void*> d_Fb, d_accb;
  void* d_F = nullptr;          // complex T [ncols][Lpad]
  void* d_X = nullptr;          // complex T [nrows][ncols]
  void* d_G = nullptr;          // complex T [nrows][gstride]
  void* d_sT = nullptr;         // T [2L-1], deconvolution in Theta incl. 1/(2L), n = -(L-1)..L-1
  void* d_sP = nullptr;         // T [2M+1], deconvolution in phi, m = -M..M
  void* d_w = nullptr;          // T [nring]
  void* d_tw2L = nullptr;       // complex T twiddles e^{-2 pi i t/N}
  void* d_tw4L = nullptr;
  void* d_twP = nullptr;
  FftDev f2L{}, f4L{}, fP{};
  int* d_perm2L = nullptr;      // digit-reversed positions of each FFT length
  int* d_perm4L = nullptr;
  int* d_permP = nullptr;
  void* d_fscratch = nullptr;   // global FFT buffers for lengths beyond shared memory (else null)
  // points (sorted by tile)
  TileItem* d_titems = nullptr;
  int* d_roff = nullptr;        // FP32 form: first sorted point of each (tile, base row), ntr ntq TR + 1 entries
  int ntitems = 0;
  int32_t* d_pidx = nullptr;    // FP64 form: original index of sorted point
  int32_t* d_pcell = nullptr;   // FP64 form: (r0 - tile row origin) | (q0 + padq - tile col origin) << 16
  void* d_pw = nullptr;         // FP64 form: weights [2W][npts] (psi_r[i], then psi_q[k])
  int4* d_prec = nullptr;       // FP32 form, per sorted point: (index, cell, bits of t - r0, bits of u - q0)
  void* d_io_a = nullptr;       // device staging for the host-buffer entry points (lazy)
  void* d_io_f = nullptr;
  // host-buffer entry points: the recursions run in chunks of orders m so that the a_lm copies
  // overlap them (FP32 form); synthesis chunk k covers m in [chunk_m[k], chunk_m[k+1]) and items
  // [chunk_item[k], chunk_item[k+1]), adjoint chunks likewise from achunk_m and chunk_aitem
  std::vector<int> chunk_m, chunk_item, achunk_m, chunk_aitem;
  cudaStream_t copy_st = nullptr;
  std::vector<cudaEvent_t> chunk_ev;
  // item and order ranges of the next recursion launch (-1: all); set only around chunked launches
  int r_item0 = 0, r_item1 = -1, r_aitem0 = 0, r_aitem1 = -1, r_m0 = 0, r_m1 = -1;
  // patch-centred frame (PSHT_PATCH_FRAME): the plan's rings, grid and points live in the frame
  // rotated by euler; a_lm are rotated on the way in and back on the way out, and a spin-s map
  // picks up the basis angle of each point
  int patch = 0;
  double euler[3] = {0.0, 0.0, 0.0};
  Rotator* rot = nullptr;
  void* d_ra = nullptr;   // complex T [2][nalm], rotated a_lm
  void* d_sph = nullptr;  // complex T [npts], e^{i s psi_p} (spin > 0)
  void* d_fr = nullptr;   // complex T [npts], adjoint input in the rotated basis (spin > 0)
  size_t bytes = 0;
  std::vector<void*> allocs;
  // stage timing (psht_plan_profile)
  bool profile = false;
  struct StageRec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<StageRec> recs;
  std::vector<cudaEvent_t> evpool;
};

// Let kernel fn use at least `bytes` of dynamic shared memory.  The attribute is set once per
// kernel and device, to the most the device grants the kernel, and never lowered: a kernel whose
// dynamic size depends on the plan (the FFT stages) is launched by several host threads at once
// (the request server), and a per-launch setting lowered by one thread between another thread's
// setting and launch made that launch fail ("too many resources requested").
void allow_dynamic_smem(const void* fn, size_t bytes);

// kernels / launchers ---------------------------------------------------------------------------
int rec_table_record_bytes(int prec);  // bytes per (l, m) record of the recurrence table
void build_rec_table(Plan& p, cudaStream_t st);
// after build_rec_table: fill the start states (buffers allocated by the planner)
void build_rec_starts(Plan& p, cudaStream_t st);
// msc: weight of the m > 0 a_lm entries (read by the synthesis, written by the adjoint)
void launch_rec_synthesis(Plan& p, const void* g, const void* c, cudaStream_t st, double msc = 1.0);
void launch_rec_adjoint(Plan& p, void* g, void* c, cudaStream_t st, double msc = 1.0);
// several sets in one pass (the Wigner columns of every (ring, m, l) evaluated once for all sets):
// synthesis of a_lm sets (g[k], c[k]) into ring coefficients F[k]; adjoint of ring coefficients F[k]
// into (g[k], c[k]), the FP32 form accumulating orders with several items in acc[k] (float4[nalm],
// zero on entry and on exit).  c may be null (no c sets).
void launch_rec_synthesis_sets(Plan& p, int nsets, const void* const* g, const void* const* c, void* const* F,
                               cudaStream_t st, double msc = 1.0);
void launch_rec_adjoint_sets(Plan& p, int nsets, void* const* F, void* const* acc, void* const* g, void* const* c,
                             cudaStream_t st, double msc = 1.0);
void launch_theta_synthesis(Plan& p, cudaStream_t st);
void launch_phi_synthesis(Plan& p, cudaStream_t st);
void launch_phi_adjoint(Plan& p, cudaStream_t st);
void launch_theta_adjoint(Plan& p, cudaStream_t st);
void launch_gather(Plan& p, void* f, cudaStream_t st);
void launch_scatter(Plan& p, const void* f, cudaStream_t st);
void launch_ring_coeffs_export(Plan& p, void* F, cudaStream_t st);
void reduce_points(const double* theta, const double* phi, int64_t npts, double out[3], cudaStream_t st);
void bin_points(Plan& p, const double* theta, const double* phi, cudaStream_t st);
int max_fft_len(int prec);                // longest FFT held in one CTA's shared memory
size_t fft_scratch_elems(const Plan& p);  // complex elements of the global FFT buffers (0: none)
void ring_synthesis_noalloc(int spin, int lmax, const double* theta, int nring, const void* g, const void* c, void* F,
                            cudaStream_t st);
size_t noalloc_scratch_bytes();
// predicted relative rms error of the plan's ring set for spectrum cl at angles beta (host arrays)
void predict_error_device(const Plan& p, const std::vector<MSeed>& seeds, const double* cl, const double* beta, int n,
                          double* rel_rms, cudaStream_t st);

// change of frame (psht_rotate.cu): Wigner-D rotation of a_lm sets through d(pi/2), rotation of
// points with the spin-basis angle, and the rotation that centres the points' smallest cap on the pole
Rotator* rotator_create(int lmax, int prec, cudaStream_t st);
void rotator_destroy(Rotator* r);
// in_msc weighs the m > 0 inputs, out_msc the m > 0 outputs
void rotator_apply(Rotator& r, double alpha, double beta, double gamma, const void* g, const void* c, void* go,
                   void* co, cudaStream_t st, double in_msc = 1.0, double out_msc = 1.0);
int rotator_lmax(const Rotator* r);
int rotator_prec(const Rotator* r);
size_t rotator_bytes(int lmax, int prec);
void rotate_points_device(double alpha, double beta, double gamma, const double* theta, const double* phi,
                          int64_t n, double* theta2, double* phi2, double* psi, cudaStream_t st);
void patch_rotation_device(const double* theta, const double* phi, int64_t n, double euler[3], double* theta_star,
                           cudaStream_t st);
void spin_phase_device(int prec, const double* psi, int s, int64_t n, void* ph, cudaStream_t st);
void mul_phase_device(int prec, const void* in, const void* ph, int64_t n, bool conj, void* out, cudaStream_t st);

}  // namespace psht
