/*
 * psht.h -- C ABI of the GB300 (sm_103a) partial-sky spin-s spherical harmonic transforms.
 *
 * The library computes the two operations that open Carron & Reinecke, "Fast partial-sky
 * spherical harmonic transforms" (Sec. I):
 *
 *   synthesis general       f_p = - sum_{l<=lmax} sum_{|m|<=l} (g_lm + i c_lm) sY_lm(theta_p, phi_p)
 *   adjoint synthesis general
 *       g~_lm = -1/2    sum_p [ f_p sY*_lm(theta_p, phi_p) + (-1)^s f*_p _{-s}Y*_lm(theta_p, phi_p) ]
 *       c~_lm = -1/(2i) sum_p [ f_p sY*_lm(theta_p, phi_p) - (-1)^s f*_p _{-s}Y*_lm(theta_p, phi_p) ]
 *
 * with sY_lm(theta, phi) = sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi} (appendix, eq. Ylm), by the
 * partial-sky Fourier-sphere route (Sec. II, steps 1-4): a Wigner-d recursion onto the few apodised
 * rings that cover the patch, FFTs onto an oversampled reduced Fourier grid, and ES-kernel
 * interpolation (gather) or spreading (scatter-add) at the points.
 *
 * Conventions shared by every entry point
 *   a_lm    packed m-major, idx(l, m) = m(2 lmax + 1 - m)/2 + l for 0 <= m <= l <= lmax,
 *           (lmax+1)(lmax+2)/2 complex values, interleaved (re, im); complex128 in the FP64 form,
 *           complex64 in the FP32 form.  The negative orders follow the reality rule
 *           a_{l,-m} = (-1)^m a*_lm for g and c separately (Sec. I).  On input Im(a_l0) and l < s
 *           are ignored; on output they are written as 0.
 *   f       npts complex values, interleaved, complex128 (FP64 form) or complex64 (FP32 form).
 *   points  theta, phi: npts float64 values in every form; theta in [0, pi], phi any finite value.
 *   streams every device-side call enqueues all its work on `stream` (a cudaStream_t passed as
 *           void*, NULL = legacy default stream) and returns without synchronising, except where
 *           stated.  Pointers marked DEVICE must be device (or managed) memory owned by the caller;
 *           the library never frees caller memory.
 *   errors  0 on success, a negative PSHT_E* code on failure; psht_last_error() then returns a
 *           message for the calling thread.  Failed calls leave caller buffers unspecified but
 *           never write outside them.  Arguments are validated on the host before any launch.
 */
#ifndef PSHT_H
#define PSHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSHT_OK 0
#define PSHT_EINVAL (-22)   /* bad argument (sizes, spin, eps, NaN or out-of-range theta, ...) */
#define PSHT_ENOMEM (-12)   /* device allocation failed or above the plan's memory budget      */
#define PSHT_ECUDA (-5)     /* a CUDA runtime call failed                                       */
#define PSHT_ENOTSUP (-95)  /* configuration outside what this build supports (message says why) */

/* precision / option flags for psht_plan_create */
#define PSHT_AUTO 0u        /* FP32 form for eps >= 1e-5, FP64 form below                       */
#define PSHT_FP64 1u        /* FP64 everywhere                                                   */
#define PSHT_FP32 2u        /* FP32 recursion (FP64 seeds and rescaling), FP32 FFT and kernels;  */
                            /* eps >= 1e-6 only (below it the FP64 form is required)             */
#define PSHT_FULL_SKY 4u    /* full-sky route whatever the points' extent (Sec. I: theta_max = pi, */
                            /* w = 1, Lmax = lmax); the baseline of the paper's speed-ups (Table 1) */
#define PSHT_PATCH_FRAME 8u /* run in the patch-centred frame (Sec. II step 1): the plan rotates the */
                            /* points so that the centre of their smallest cap is the north pole    */
                            /* (psht_patch_rotation), rotates a_lm in (and the adjoint's a_lm back)  */
                            /* with psht_rotator_apply, and applies each point's basis angle to     */
                            /* spin-s values; inputs and outputs stay in the caller's frame         */

typedef struct psht_plan psht_plan; /* opaque; owned by the library, freed by psht_plan_destroy */

/* Plan parameters, filled by psht_plan_info.  Names follow the paper (Sec. II). */
typedef struct psht_info {
  int spin, lmax, precision;     /* precision: 64 or 32                                        */
  int pole;                      /* +1: north pole used, -1: south pole (Sec. II step 1)       */
  int full_sky;                  /* 1 when theta_max >= pi or Lmax >= lmax (no apodisation)    */
  double eps, theta_star, eps_apo, theta_max, alpha, dTheta;
  int Lmax, L, nring;            /* rings Theta_j = j pi/L, j < nring                         */
  int M;                         /* phi band limit after polar optimisation                    */
  int W;                         /* ES kernel width (cells)                                    */
  double beta_es;                /* ES kernel shape                                            */
  int nTheta, nphi;              /* oversampled grid; nTheta = 4L                              */
  int r_lo, nrows;               /* grid rows kept: r_lo .. r_lo + nrows - 1                   */
  int64_t npts;
  int64_t ring_mode_pairs;       /* (ring, m) pairs the recursion computes                    */
  int64_t recursion_triples;     /* (ring, m, l) steps of the recursion                       */
  size_t device_bytes;           /* device memory held by the plan                             */
  int patch_frame;               /* 1: PSHT_PATCH_FRAME (theta_star etc. refer to that frame)  */
  double euler[3];               /* its rotation (alpha, beta, gamma), as psht_patch_rotation  */
} psht_info;

/*
 * Create a plan for synthesis/adjoint at fixed points (Sec. II steps 1-4, parameter choice of
 * Sec. II.C-D).  theta, phi: DEVICE float64[npts], read during this call only.  Synchronises
 * `stream` once (theta* reduction and point binning).  Returns PSHT_EINVAL for spin < 0,
 * lmax < spin, eps outside [1e-14, 1e-1], PSHT_FP32 with eps < 1e-6, npts < 0, NaN/out-of-range
 * theta or non-finite phi;
 * PSHT_ENOMEM if the plan does not fit in device memory.  *out receives the plan.
 */
int psht_plan_create(int spin, int lmax, const double* theta, const double* phi, int64_t npts, double eps,
                     uint32_t flags, void* stream, psht_plan** out);

/* Copy the plan's parameters into *info (host memory).  Never fails for a valid plan. */
int psht_plan_info(const psht_plan* plan, psht_info* info);


/*
 * Synthesis general (Sec. I eq. syn) at the plan's points.  g, c: DEVICE packed a_lm (c may be
 * NULL: c = 0); f: DEVICE output, npts complex values in the caller's point order.
 * Overwrites f entirely.  Concurrent calls on one plan must use the same stream (the plan's
 * work buffers are reused).
 */
int psht_plan_synthesis(psht_plan* plan, const void* g, const void* c, void* f, void* stream);

/*
 * Adjoint synthesis general (Sec. I) at the plan's points: the exact transpose of
 * psht_plan_synthesis for <f, f'> = Re sum_p conj(f_p) f'_p and <a, a'> = sum_l sum_{|m|<=l}
 * Re(conj(a_lm) a'_lm) summed over g and c.  f: DEVICE input; g: DEVICE output (required);
 * c: DEVICE output or NULL (then c~ is not written).  Overwrites g and c entirely.
 */
int psht_plan_adjoint(psht_plan* plan, const void* f, void* g, void* c, void* stream);

/*
 * Plan options beyond the paper's argument list (psht_plan_create_ex).  Zero-initialise the struct:
 * zero fields take the defaults.
 *   window: the bell of the apodisation window (Sec. II.D): PSHT_WINDOW_ES, the exponential of a
 *     semicircle the paper settles on (default), or PSHT_WINDOW_KB, the Kaiser-Bessel bell
 *     I0(|ln eps| sqrt(1 - v^2)) the paper compares it with; same support and shape parameter.
 *   kappa: factor on the Fourier-sphere band limit, Lmax = ceil(kappa (lmax theta_star / pi)(1+eps_apo)^2)
 *     (Sec. II.C); 0 means 1.  Below 1 the ring count shrinks and the error grows beyond eps
 *     unless the field is smooth (psht_predict_error tells by how much).
 */
#define PSHT_WINDOW_ES 0
#define PSHT_WINDOW_KB 1
#define PSHT_APO_PAPER 0    /* eps_apo = sqrt(2 |ln eps| / (theta_star lmax)), minimising Lmax (eq. Lmax2)  */
#define PSHT_APO_COST 1     /* eps_apo minimising the recursion's (ring, m, l) count with polar          */
                            /* optimisation, the alternative the paper mentions beside eq. Lmax2        */
typedef struct {
  int window;
  double kappa;
  /* apodisation: PSHT_APO_PAPER (default) or PSHT_APO_COST.  With PSHT_APO_COST the planner tries
   * eps_apo = e0 (20 + k)/40, k = 0..80 (e0 the paper's value), with the band limit the window needs
   * for that apodisation length, Lmax = ceil(kappa (lmax theta_star / pi)(1 + eps_apo)(1 + e0^2/eps_apo))
   * (the paper's Lmax before minimisation over eps_apo), and keeps the cheapest. */
  int apodisation;
} psht_options;
/* psht_plan_create with options; opt may be NULL (defaults). */
int psht_plan_create_ex(int spin, int lmax, const double* theta, const double* phi, int64_t npts, double eps,
                        uint32_t flags, const psht_options* opt, void* stream, psht_plan** out);

/*
 * The planner alone (Sec. II steps 2-4, II.C-D), on the host, for a given theta_star about the
 * north pole: fills *info as psht_plan_info would for a plan of npts = 0 (device_bytes: the
 * estimate for no points), and, where not NULL, the rings' colatitudes theta_j, window weights w_j
 * and polar cutoffs Mj (HOST arrays of info->nring entries: call once with NULL to learn nring).
 * opt may be NULL.  No device work.  EINVAL for invalid arguments.
 */
int psht_plan_params(int spin, int lmax, double theta_star, double eps, uint32_t flags, const psht_options* opt,
                     psht_info* info, double* theta_j, double* w_j, int32_t* Mj);

/*
 * Predicted error of the partial-sky route for a statistically isotropic field (Sec. II.E):
 * c_m = sum_l C_l (2l+1)/2 |d^l_{m,-s}(pi/2)|^2 (eq. cm, eq. cms), the error of each wave e^{i m theta}
 * after weighting and band limiting on the plan's rings, sigma_m^2(theta) (eq. s2m), and
 * sigma^2(theta) = (1/2pi) sum_m c_m sigma_m^2(theta) (eq. st), returned relative to the field's
 * variance (1/2pi) sum_m c_m as an rms ratio.  The ring set is the one psht_plan_create_ex would
 * build for (spin, lmax, theta_star, eps, opt); the NUFFT's own error is not included.
 *   cl: HOST double[lmax+1], C_l (spin 0) or C^E_l + C^B_l (spin > 0); beta: HOST double[n], angular
 *   distances from the plan's pole at which to predict; rel_rms: HOST double[n] output.
 * Runs on the current device, synchronising `stream`.  EINVAL for bad sizes or negative C_l.
 */
int psht_predict_error(int spin, int lmax, double theta_star, double eps, const psht_options* opt, const double* cl,
                       const double* beta, int n, double* rel_rms, void* stream);

/*
 * Batched forms: nsets independent transforms on one plan, with the same results as nsets calls of
 * psht_plan_synthesis / psht_plan_adjoint.  Up to 4 sets share one pass of the Wigner-d recursion
 * (the recursion's columns of every (ring, m, l) are evaluated once and applied to each set: the
 * recursion costs about 1.5-2.5x a single set's for 4 sets instead of 4x); the FFT, interpolation
 * and spreading stages run set by set.  g, c, f: HOST arrays of nsets DEVICE pointers, laid out as
 * for the single-set calls; c may be NULL (c = 0 for every set in the synthesis, no c~ in the
 * adjoint) or hold NULL entries.  nsets in [1, PSHT_MAX_BATCH]; larger batches run in groups of 4.
 * The first call with more than one set allocates device buffers for 3 extra sets (ring
 * coefficients, and in the FP32 form an accumulator of 16 B per coefficient each), which the plan
 * keeps (psht_plan_info's device_bytes includes them from then on).  A PSHT_PATCH_FRAME plan runs
 * the sets one after the other.  Asynchronous on `stream`; errors as for the single-set calls.
 */
#define PSHT_MAX_BATCH 64
int psht_plan_synthesis_batch(psht_plan* plan, int nsets, const void* const* g, const void* const* c, void* const* f,
                              void* stream);
int psht_plan_adjoint_batch(psht_plan* plan, int nsets, const void* const* f, void* const* g, void* const* c,
                            void* stream);

/*
 * Packed-gradient forms, for automatic differentiation over the packed a_lm arrays.  The transpose
 * above pairs with the inner product that counts each m > 0 entry twice (it stands for m and -m,
 * eq. syn's reality condition), while a gradient over the packed storage counts every stored
 * entry once: dL/dRe a + i dL/dIm a for a real loss L.
 *   psht_plan_adjoint_packed: as psht_plan_adjoint, with the m > 0 entries of g~ and c~ doubled,
 *     i.e. the packed gradients of Re sum_p conj(f_p) [synthesis(g, c)]_p with respect to g and c.
 *   psht_plan_synthesis_packed: as psht_plan_synthesis, with the m > 0 entries of g and c halved,
 *     i.e. the gradient with respect to f of Re <(g, c), adjoint(f)> taken over the packed storage.
 * m = 0 entries are unchanged (their imaginary parts are ignored on input and written as 0).
 * Arguments, layout, ownership and errors as for the plain forms.
 */
int psht_plan_synthesis_packed(psht_plan* plan, const void* g, const void* c, void* f, void* stream);
int psht_plan_adjoint_packed(psht_plan* plan, const void* f, void* g, void* c, void* stream);

/*
 * Host-buffer forms of the two calls above: g, c, f are HOST pointers (pinned memory gives the
 * fastest copies).  Copies inputs to the device, runs the transform on `stream` and copies the
 * result back; returns after `stream` has synchronised, so the host buffers hold the result.
 */
int psht_plan_synthesis_host(psht_plan* plan, const void* g, const void* c, void* f, void* stream);
int psht_plan_adjoint_host(psht_plan* plan, const void* f, void* g, void* c, void* stream);

/*
 * Device status of the plan: synchronises `stream` and writes 0 to *status if every kernel wait of
 * earlier calls completed, or 1 if a wait on an asynchronous copy gave up after its iteration
 * limit (the kernel then stopped early and the call's outputs are invalid).  Clears the word.
 */
int psht_plan_status(psht_plan* plan, int* status, void* stream);

/* Release the plan and all device memory it holds.  Synchronises the device. NULL is a no-op. */
int psht_plan_destroy(psht_plan* plan);

/*
 * Diagnostic stage access, used by the stage-parity tests.
 *   psht_plan_rings: the planner's ring table, HOST outputs theta_j[nring], w_j[nring],
 *     Mj[nring] (int32), any of them may be NULL.
 *   psht_plan_ring_coeffs: ring Fourier coefficients F_j[m] = -sum_l (g+ic)_lm N_l d^l_{m,-s}(theta_j)
 *     (Sec. II step 4 applied to the rings), DEVICE output F[nring][2M+1] (m + M fastest),
 *     complex in the plan's precision; zero where |m| > M_j.
 */
int psht_plan_rings(const psht_plan* plan, double* theta_j, double* w_j, int32_t* Mj);
int psht_plan_ring_coeffs(psht_plan* plan, const void* g, const void* c, void* F, void* stream);

/*
 * Stage timing.  psht_plan_profile(plan, 1) makes every later execute call record CUDA events on
 * its stream around each stage (0 recursion, 1 Theta FFT, 2 phi FFT, 3 gather; adjoint: 4 scatter
 * incl. grid clearing, 5 phi FFT, 6 Theta FFT, 7 recursion); 0 stops recording.
 * psht_plan_stage_times synchronises the recorded events and writes, per stage, the summed
 * milliseconds into ms[PSHT_NSTAGES] and the number of launches into calls[PSHT_NSTAGES] (either may
 * be NULL), then clears the record.
 */
#define PSHT_NSTAGES 8
int psht_plan_profile(psht_plan* plan, int enable);
int psht_plan_stage_times(psht_plan* plan, double* ms, int64_t* calls);

/*
 * One-shot forms with the paper's argument list (g, c, spin, lmax, theta, phi, eps): plan,
 * execute and destroy.  All pointers DEVICE.  Precision PSHT_AUTO.  Synchronise `stream`.
 */
int psht_synthesis(const void* g, const void* c, int spin, int lmax, const double* theta, const double* phi,
                   int64_t npts, double eps, void* f, void* stream);
int psht_adjoint_synthesis(const void* f, int spin, int lmax, const double* theta, const double* phi,
                           int64_t npts, double eps, void* g, void* c, void* stream);

/*
 * Allocation-free ring synthesis.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory — their device memory is owned by another allocator
 * (a framework's caching pool, a memory-capped service), or they must not call cudaMalloc/cudaFree,
 * which can synchronise the whole device, inside their own work.
 *
 * It computes the ring Fourier coefficients of synthesis general at arbitrary ring colatitudes,
 *   F[j][m + lmax] = -sum_l (g_lm + i c_lm) sqrt((2l+1)/4pi) d^l_{m,-s}(theta_j),  |m| <= lmax,
 * (the quantity psht_plan_ring_coeffs returns for a plan's rings, without the polar cutoff), in
 * FP64, without a plan and without allocating: every intermediate lives in one fixed device array
 * of the library (psht_noalloc_scratch_bytes(), about 4.4 MB), which every GPU that loads the
 * library holds until the process exits.
 *   theta: DEVICE float64[nring] in [0, pi];  g, c: DEVICE packed complex128 a_lm (c may be NULL);
 *   F: DEVICE complex128 output [nring][2 lmax + 1], fully written.
 * Limits: lmax <= PSHT_NOALLOC_MAX_LMAX, nring <= PSHT_NOALLOC_MAX_RINGS; larger sizes return
 * PSHT_EINVAL with a message.  The array is shared by all calls and keeps the last call's contents
 * (each call rewrites all it uses); calls that overlap on the GPU race on it and must be ordered
 * by the caller.  The first call on a device looks up the array's address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  Asynchronous on
 * `stream`.
 */
#define PSHT_NOALLOC_MAX_LMAX 511
#define PSHT_NOALLOC_MAX_RINGS 4096
int psht_ring_synthesis_noalloc(int spin, int lmax, const double* theta, int nring, const void* g, const void* c,
                                void* F, void* stream);
size_t psht_noalloc_scratch_bytes(void);

/*
 * Change of frame.  The paper evaluates its rings about a pole placed at the centre of the patch
 * (Sec. II, step 1) and leaves the rotation of a caller's coefficients to them.  These entry points
 * rotate a_lm sets, points and the spin basis between frames.
 *
 * A rotation is given by zyz Euler angles, R = R_z(alpha) R_y(beta) R_z(gamma) acting on vectors.
 * Rotating one real field's coefficient set (g or c, packed m-major as everywhere in this header):
 *   a'_lm = sum_{m'=-l..l} e^{-i m alpha} d^l_{m m'}(beta) e^{-i m' gamma} a_lm',  m >= 0,
 * with a_{l,-m'} = (-1)^m' a*_lm' and d^l the appendix's Wigner small-d (eq. Ylm).  A spin-s map
 * synthesised from the rotated (g', c') at the rotated point n = R p equals the original map at p up
 * to the change of local basis: f(p) = e^{i s psi_p} f'(R p), psi_p from psht_rotate_points.  The
 * inverse rotation is (-gamma, -beta, -alpha); it is also the adjoint, since D^l is unitary for the
 * inner product of the adjoint synthesis (sum over all m of Re(a* a')).
 *
 * The library evaluates d^l(beta) through d^l(pi/2) by the appendix's Fourier identity
 * d^l_{m m'}(beta) = sum_k i^m d^l_{km}(pi/2) e^{-i k beta} d^l_{km'}(pi/2) (-i)^m', with
 * d^l(pi/2) generated on the fly by a recurrence, in O(lmax^3) work and no O(lmax^2) table beyond
 * one coefficient per (l, m').  Precision PSHT_FP64 (complex128 sets) or PSHT_FP32 (complex64 sets;
 * relative error a few 1e-6 at lmax 4096, growing slowly with lmax); PSHT_AUTO means PSHT_FP64.
 *
 * psht_rotator_create: the per-band-limit tables and scratch (psht_rotator_bytes); asynchronous on
 *   `stream`.  psht_rotator_apply: rotates g (and c, if not NULL) into g_out (c_out); all DEVICE
 *   pointers of nalm = (lmax+1)(lmax+2)/2 complex elements; the output may alias the input; c and
 *   c_out are both NULL or both set.  Asynchronous on `stream`; calls on one rotator share its
 *   scratch and must be ordered.  Im of the m = 0 inputs is ignored and written as 0.
 * psht_rotate_alm: create, apply, destroy (synchronises `stream`).
 */
typedef struct psht_rotator psht_rotator;
int psht_rotator_create(int lmax, uint32_t flags, void* stream, psht_rotator** out);
int psht_rotator_apply(psht_rotator* rot, double alpha, double beta, double gamma, const void* g, const void* c,
                       void* g_out, void* c_out, void* stream);
int psht_rotator_destroy(psht_rotator* rot);
size_t psht_rotator_bytes(int lmax, uint32_t flags);
int psht_rotate_alm(int lmax, double alpha, double beta, double gamma, const void* g, const void* c, void* g_out,
                    void* c_out, uint32_t flags, void* stream);

/*
 * Synthesis and adjoint of a PSHT_PATCH_FRAME plan with the a_lm in the plan's own frame (rotated
 * by psht_plan_info's euler): no rotation on the way in or out, the points' spin-basis angle still
 * applied, so f stays in the caller's frame and basis.  An iterative solver rotates its a_lm once
 * (psht_rotator_apply with euler), iterates with these, and rotates the result back with
 * (-gamma, -beta, -alpha).  Same arguments and rules as psht_plan_synthesis / psht_plan_adjoint;
 * EINVAL for a plan without PSHT_PATCH_FRAME.
 */
int psht_plan_synthesis_inframe(psht_plan* plan, const void* g, const void* c, void* f, void* stream);
int psht_plan_adjoint_inframe(psht_plan* plan, const void* f, void* g, void* c, void* stream);

/*
 * Rotated points n_p = R p: theta_out in [0, pi], phi_out in [0, 2 pi), and (if psi_out is not NULL)
 * psi_p, the angle from e_theta(p) towards e_phi(p) of the rotated frame's e_theta at n_p carried
 * back by R^-1, so that f(p) = e^{i s psi_p} f'(n_p) for a spin-s map in the two frames.
 * All arrays DEVICE float64[npts]; outputs may alias inputs.  Asynchronous on `stream`.
 */
int psht_rotate_points(double alpha, double beta, double gamma, const double* theta, const double* phi, int64_t npts,
                       double* theta_out, double* phi_out, double* psi_out, void* stream);

/*
 * Patch-centred frame (Sec. II, step 1: coordinates whose north pole sits at the patch centre): the
 * centre c of the smallest spherical cap holding the points (the direction of the minimum-norm
 * point of their convex hull, by Wolfe's iteration with the linear minimisations on the device),
 * returned as the Euler angles euler[3] = (0, theta_c, pi - phi_c) of a rotation taking c to the
 * north pole, and (if theta_star is not NULL) the cap radius.  theta, phi: DEVICE float64[npts];
 * euler, theta_star: HOST.  Synchronises `stream`.  EINVAL for NaN, out-of-range or non-finite
 * coordinates and if the points do not lie in an open hemisphere.
 */
int psht_patch_rotation(const double* theta, const double* phi, int64_t npts, double* euler, double* theta_star,
                        void* stream);

/* Device bytes a plan for these arguments would hold (theta_star = max distance to the pole). */
size_t psht_estimate_bytes(int spin, int lmax, double theta_star, int64_t npts, double eps, uint32_t flags);

/*
 * Device bytes a plan for these points would hold: one device reduction over the points (theta*
 * and the nearer pole, Sec. II step 1), then the planner's layout.  theta, phi: DEVICE float64[npts].
 * Synchronises `stream`.  Writes *bytes; EINVAL for invalid points, as psht_plan_create.
 */
int psht_plan_estimate_points(int spin, int lmax, const double* theta, const double* phi, int64_t npts, double eps,
                              uint32_t flags, void* stream, size_t* bytes);

/*
 * Request server: a native runtime that executes many transforms concurrently on one GPU.  The
 * paper has no counterpart; it is the serving layer over the plan API above.
 *   - nstreams worker threads, each with its own non-blocking CUDA stream, take requests in
 *     arrival order; a request whose plan is in use by another worker is passed over, not waited
 *     on, so independent requests overlap on the GPU.
 *   - Continuous batching: when a worker starts a request, every request queued for the same plan
 *     and the same operation (up to 8) joins it and the group runs as one batched call
 *     (psht_plan_synthesis_batch / psht_plan_adjoint_batch), so requests that piled up while the
 *     plan was busy share its recursion pass.
 *   - Plans are cached by (points_key, npts, spin, lmax, eps, flags): the caller names its point
 *     set by points_key, and equal keys with equal npts must denote the same theta/phi values.
 *   - Admission: a new plan is created only if the cached plans plus its estimate fit in the
 *     budget (bytes; 0 = 80 % of the device memory free at creation); least-recently-used idle
 *     plans are evicted to make room; a request that cannot fit yet waits in the queue, and one
 *     that can never fit fails with PSHT_ENOMEM.
 * A request's device buffers (points, inputs, outputs) must stay valid until psht_server_wait has
 * returned for its ticket.  Latencies are host wall-clock from submission to the completion of the
 * request's stream work.
 */
#define PSHT_OP_SYNTHESIS 0
#define PSHT_OP_ADJOINT 1
typedef struct psht_server psht_server;
typedef struct {
  int op;              /* PSHT_OP_SYNTHESIS or PSHT_OP_ADJOINT                                 */
  int spin, lmax;
  double eps;
  uint32_t flags;      /* precision flags as for psht_plan_create                              */
  uint64_t points_key; /* caller's name of the point set                                       */
  const double* theta; /* DEVICE float64[npts]; read when the plan is not cached               */
  const double* phi;
  int64_t npts;
  const void* in_a;    /* synthesis: g; adjoint: f          (DEVICE, the plan's precision)     */
  const void* in_b;    /* synthesis: c or NULL; adjoint: unused                                */
  void* out_a;         /* synthesis: f; adjoint: g~                                            */
  void* out_b;         /* synthesis: unused; adjoint: c~ or NULL                               */
} psht_request;
typedef struct {
  int status;          /* PSHT_OK or the request's error code                                  */
  int worker;          /* index of the worker (stream) that ran it                             */
  int plan_cached;     /* 1 if the plan came from the cache                                    */
  int precision;       /* 32 or 64                                                              */
  double queue_ms;     /* submission to start of work                                          */
  double plan_ms;      /* plan creation (0 when cached)                                        */
  double exec_ms;      /* transform, until its stream completed                                */
  double total_ms;     /* submission to completion                                             */
  int batch;           /* requests in the batched call this request ran in (1: alone)          */
  char message[192];   /* on failure, the library's message for it ("" on success)             */
} psht_result;
typedef struct {
  int64_t submitted, completed, failed, plans_created, cache_hits, evictions;
  size_t budget, bytes_in_use, bytes_peak;
  int64_t batches;           /* plan calls made (a batch of several requests counts once)        */
  int64_t batched_requests;  /* requests that ran in a batch of more than one                    */
} psht_server_stats;

/* Start nstreams (1..64) workers on the current device.  *out receives the server. */
int psht_server_create(int nstreams, size_t budget_bytes, psht_server** out);
/* Largest batch the workers form (1..8, default 8; 1 runs every request alone).  Takes effect for
 * requests started after the call. */
int psht_server_set_batch_limit(psht_server* server, int max_batch);
/* Queue a request (copied); *ticket identifies it for psht_server_wait. */
int psht_server_submit(psht_server* server, const psht_request* request, int64_t* ticket);
/* Block until the ticket's request has finished; writes its result.  Each ticket is waited once. */
int psht_server_wait(psht_server* server, int64_t ticket, psht_result* result);
int psht_server_get_stats(psht_server* server, psht_server_stats* stats);
/* Finish every queued request, stop the workers and release all cached plans.  NULL is a no-op. */
int psht_server_destroy(psht_server* server);

/* Message of the last failing call on this thread ("" if none). */
const char* psht_last_error(void);

/* Library version string. */
const char* psht_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSHT_H */
