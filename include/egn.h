/*
 * egn.h -- C ABI of the GB300 (sm_103a) ISRS EGN nonlinear-interference integrator.
 *
 * The library evaluates, for every channel of interest (COI) n of a WDM link,
 *
 *   P_NLI,n = sum over islands (n1, n2, n3) of P_n1 P_n2 P_n3 *
 *             [ D + Phi_n1 d(n1,n3) E + Phi_n2 d(n2,n3) F + Phi_n1 d(n1,n2) G
 *               + Psi_n1 d(n1,n2) d(n2,n3) H ]                    (Eq. 15)
 *   eta_n   = P_NLI,n / P_n^3                                       (Eq. 11)
 *
 * where D..H are the 2-D (f1, f2) island integrals of Eq. 17-21 at f = the COI
 * centre, the link function Upsilon is Eq. 22 with the segment closed form of
 * the ISRS four-wave-mixing efficiency mu_s (Eq. 7-10) and the ISRS power
 * profile of Eq. 25.  The islands are the (kappa1, kappa2, l) set of Eq. 16,
 * generalised to arbitrary channel centres and rates.  Equations refer to
 * arXiv 2412.11614 (Xia et al., "Acceleration and Parallelization Methods for
 * ISRS EGN Model").
 *
 * Conventions
 *   - Units at the boundary are SI, except the customary fibre units named in
 *     egn_span.  Internally: THz, ps, km, W.
 *   - Channel centres must be strictly increasing, with supports
 *     R_n (1 + rolloff) that do not overlap.
 *   - The spectral centre f_c = (f_min + f_max) / 2 of the channel centres is
 *     the origin of the ISRS profile (Eq. 25) and of beta2/beta3 (Eq. 24);
 *     B_tot = (f_max - f_min) N / (N - 1) (B_tot = R for one channel);
 *     P_tot = sum of the launch powers.
 *   - Spans: every span is restored by an ideal amplifier (the gain/ISRS
 *     products of Eq. 22 equal 1).  Identical spans use the closed-form
 *     phased-array sum of Eq. 22; a link whose spans differ (at most 64
 *     spans) sums Eq. 22 span by span with one mu per span type and the
 *     accumulated dispersion phase.
 *   - Pulse spectra: raised cosine |S(f)|^2 = h(f)/R^2 with roll-off
 *     `rolloff`; the COI integral over f is R times the value at the COI
 *     centre (white NLI over the channel).
 *
 * Ownership: every input array is copied; the caller keeps ownership.  Host
 * outputs are caller-allocated arrays of n_ch doubles.  An egn_link owns its
 * device tables (cudaMalloc on the current device at egn_set_wdm) until
 * egn_link_destroy.
 *
 * Errors: every entry point returns an egn_status; nothing is thrown across the
 * ABI.  egn_last_error() returns a thread-local message for the last failure.
 * A link is not thread-safe: calls on one link must be serialised by the caller.
 * A failed call leaves the link usable: a failed allocation keeps the previous
 * buffer, tables whose upload failed are rebuilt by the next call, and a failed
 * egn_set_wdm leaves the link in the "no WDM set" state (EGN_E_STATE until the
 * next successful egn_set_wdm).
 *
 * Fault injection (testing the error paths without a device fault): while the
 * environment variable EGN_FAULT holds a comma-separated subset of
 *   alloc   every device and pinned host allocation fails    -> EGN_E_NOMEM
 *   h2d     every host-to-device copy fails                  -> EGN_E_CUDA
 *   launch  every evaluation's launch sequence fails          -> EGN_E_CUDA
 * the failure is returned before anything reaches the device.  The variable is
 * read on every call.
 */
#ifndef EGN_H
#define EGN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct egn_link egn_link; /* opaque, library-owned */

typedef enum {
    EGN_OK = 0,
    EGN_E_INVALID_ARG = 1, /* NULL pointer, NaN, non-positive rate/length/alpha, Cr < 0,
                              unsorted or overlapping channels, bad option value */
    EGN_E_UNSUPPORTED = 2, /* a valid request outside what this build evaluates */
    EGN_E_NOMEM = 3,       /* host or device allocation failed */
    EGN_E_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    EGN_E_TIMEOUT = 5,     /* the device did not finish within opts->timeout_ms */
    EGN_E_STATE = 6,       /* call out of order (e.g. egn_nli_eta before egn_set_wdm) */
    EGN_E_CAPACITY = 7     /* caller workspace smaller than egn_workspace_size() */
} egn_status;

/* One fibre span (Table I / Table II quantities).
 *   alpha_db_per_km   power attenuation [dB/km], > 0
 *   D_ps_nm_km        dispersion at lambda_ref_m [ps/nm/km]
 *   S_ps_nm2_km       dispersion slope at lambda_ref_m [ps/nm^2/km]
 *   lambda_ref_m      reference wavelength of D and S [m], > 0
 *   gamma_per_w_km    nonlinear coefficient [1/W/km], >= 0
 *   cr_per_w_km_thz   Raman gain slope Cr [1/W/km/THz], >= 0 (Eq. 25)
 *   length_m          span length L_s [m], > 0
 * beta2 = -D lambda^2 / (2 pi c), beta3 = (lambda^2 / (2 pi c))^2 (S + 2 D / lambda),
 * and beta2 is moved to the spectral centre by beta2 + 2 pi beta3 (f_c - c/lambda). */
typedef struct {
    double alpha_db_per_km;
    double D_ps_nm_km;
    double S_ps_nm2_km;
    double lambda_ref_m;
    double gamma_per_w_km;
    double cr_per_w_km_thz;
    double length_m;
} egn_span;

enum {
  EGN_MU_SEGMENT = 0,   /* segment closed form, Eq. 7-10 (both precisions) */
  EGN_MU_MACLAURIN = 1, /* Maclaurin closed form, Eq. 4-6 (FP64 only) */
  EGN_MU_INTEGRAL = 2   /* numerical integral of Eq. 23, the reference form (FP64 only) */
};
enum { EGN_PREC_FP64 = 0, EGN_PREC_FP32C = 1 };
enum { EGN_TERMS_GN = 0, EGN_TERMS_EGN = 1 };
enum { EGN_FMT_GAUSS = 0, EGN_FMT_QPSK = 1, EGN_FMT_16QAM = 2, EGN_FMT_64QAM = 3 };

/* Evaluation options.
 *   gl_order    n: each island is integrated with an n x n Gauss-Legendre rule
 *               (outer range split at the kinks of the inner limits into P <= 3
 *               panels of ceil(n/P) nodes, n inner nodes); 1 <= n <= 128.
 *   dz_km       segment length bound Delta z [km]: K = ceil(L / dz) segments of
 *               length L/K per span (Sec. II-C-2); K <= 1024.
 *   mu_form     EGN_MU_SEGMENT (Eq. 7-10, segments of length L/K), or, with
 *               EGN_PREC_FP64 only, EGN_MU_MACLAURIN (Eq. 4-6) or
 *               EGN_MU_INTEGRAL (Eq. 23 integrated numerically: 10-point
 *               Gauss-Legendre on equal pieces of at most a quarter period
 *               pi / (2 |chi|) of the phase factor; dz_km is then unused but
 *               must be valid).  Other combinations: EGN_E_UNSUPPORTED.
 *   precision   EGN_PREC_FP64: every step in FP64 (the plain baseline);
 *               EGN_PREC_FP32C: FP32 integrand, phases reduced exactly with
 *               FP64 island constants and compensated FP32 (double-float)
 *               arithmetic, compensated island sums.
 *   terms       EGN_TERMS_GN (D only) or EGN_TERMS_EGN (D + E, F, G, H).
 *   timeout_ms  host-side wait limit for egn_nli_eta (0 = none) -> EGN_E_TIMEOUT.
 *               The queued work then still runs to completion on `stream`; the
 *               outputs are not written; the link stays valid and a later call
 *               on the same stream is ordered after the timed-out work.
 *   stream      cudaStream_t to launch on (NULL = the legacy default stream). */
typedef struct {
    int gl_order;
    double dz_km;
    int mu_form;
    int precision;
    int terms;
    int timeout_ms;
    void* stream;
} egn_opts;

/* Create a link from n_spans >= 1 spans (copied).  Returns EGN_E_INVALID_ARG on
 * bad parameters.  Identical spans use the phased-array closed form of Eq. 22;
 * spans that differ (fibre or length) use the explicit coherent sum of Eq. 22
 * for up to 64 spans (longer heterogeneous links are refused by the evaluation
 * calls with EGN_E_UNSUPPORTED).  Up to 4 distinct span types evaluate each
 * type's mu once per point with shared-memory c_k tables (their segments
 * together at most 880); more types walk the spans in order, forming c_k on the
 * fly, and egn_nli_eta_static refuses them (EGN_E_UNSUPPORTED). */
egn_status egn_link_create(const egn_span* spans, int n_spans, egn_link** out);

/* Release the link and its device tables.  NULL is ignored. */
void egn_link_destroy(egn_link* link);

/* Set the WDM comb (Eq. 15-16 inputs).  n_ch >= 1 channels with centre
 * frequencies [Hz] (strictly increasing, non-overlapping supports), symbol rates
 * [Baud], launch powers [W] (> 0), EGN modulation constants Phi and Psi per
 * channel (see egn_format_moments), raised-cosine roll-off in [0, 1].
 * Uploads the channel table to the current device and counts the islands on it
 * (synchronously, on the legacy default stream): work of egn_nli_eta_device on
 * another stream that still reads this link must have completed.  Combs with
 * more than 2^32 - 1 islands -> EGN_E_UNSUPPORTED (32-bit island indices).
 * Mixed symbol rates with any Phi or Psi != 0 -> EGN_E_UNSUPPORTED (the paper
 * gives the correction terms for one symbol rate only). */
egn_status egn_set_wdm(egn_link* link, int n_ch, const double* centre_hz, const double* symbol_rate_baud,
                       const double* launch_power_w, const double* phi, const double* psi, double rolloff);

/* Bytes of device workspace egn_nli_eta_device needs for these options. */
egn_status egn_workspace_size(const egn_link* link, const egn_opts* opts, size_t* bytes);

/* Number of islands of the current comb: total, and per COI if per_coi != NULL
 * (n_ch entries).  Every island (n1, n2, n3) has a mirror (n2, n1, n3) under
 * f1 <-> f2 with the same D, so the integrator evaluates only the islands with
 * n1 <= n2 (*n_half); *n_e and *n_f are the sizes of the E list (n1 == n3,
 * n1 <= n2) and of the F list (n2 == n3, n1 < n2).  Any output may be NULL. */
egn_status egn_island_count(const egn_link* link, long long* total, long long* per_coi, long long* n_half,
                            long long* n_e, long long* n_f);

/* eta_n [1/W^2] and P_NLI,n [W] for every channel into caller host arrays of
 * n_ch doubles (either may be NULL).  Synchronous: plans the islands on the
 * device, integrates, assembles, copies back.  Uses a library-owned device
 * workspace that is kept between calls. */
egn_status egn_nli_eta(egn_link* link, const egn_opts* opts, double* eta_per_w2, double* pnli_w);

/* The same with the integral over f of Eq. 17-21 taken literally instead of
 * the white-NLI value R_n G(f_n): P_NLI,n = int over f in [f_n - R_n/2,
 * f_n + R_n/2] of G(f) df by an n_f-point Gauss-Legendre rule (1 <= n_f <= 64),
 * G(f) the 2-D island integral (Eq. 15 with D..H at COI frequency f divided by
 * R_n), so P_NLI,n = sum_j (w_j / 2) P_NLI,n(f_n + x_j R_n / 2).  Every node is a
 * full evaluation (islands planned for that f, all opts as for egn_nli_eta);
 * n_f = 1 equals egn_nli_eta.  Synchronous; eta and pnli are host arrays of
 * n_ch doubles (either may be NULL).  Cost: n_f evaluations. */
egn_status egn_nli_eta_3d(egn_link* link, const egn_opts* opts, int n_f, double* eta_per_w2, double* pnli_w);

/* Device variant: same computation, asynchronous on opts->stream, writing
 * eta_dev and pnli_dev (device arrays of n_ch doubles, either may be NULL) and
 * using the caller's device workspace of at least egn_workspace_size() bytes
 * (256-byte aligned).  Returns after the launches; errors found on the device
 * are reported by the next call. */
egn_status egn_nli_eta_device(egn_link* link, const egn_opts* opts, void* workspace, size_t workspace_bytes,
                              double* eta_dev, double* pnli_dev);

/* Evaluation that allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- an application whose
 * device memory is owned by another allocator (a framework's caching allocator or
 * a pool sized up front on a shared GPU), a control loop that re-evaluates links
 * online and cannot take the device synchronisation of cudaMalloc/cudaFree, or a
 * plugin host that forbids device allocation.  Same computation as
 * egn_nli_eta_device, asynchronous on opts->stream, writing eta_dev and pnli_dev
 * (device arrays of n_ch doubles, both required).  Its scratch (link tables and
 * workspace) is one 16 MiB array compiled into the library, which every GPU that
 * loads the library holds until the process exits; an evaluation that needs more
 * (egn_workspace_size + the tables; about 60 channels at EGN_PREC_FP32C) is
 * refused with EGN_E_CAPACITY.  The link's segment and Gauss-Legendre tables
 * are formed on the device by a kernel from its launch parameters, so no host
 * buffer is read after the call returns.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the one array
 * and it keeps the last call's contents: calls whose work overlaps on the GPU
 * (other streams, other threads, other links) race and must be serialised by the
 * caller.  Host threads that make their first call on one device at the same
 * time are serialised inside the library. */
egn_status egn_nli_eta_static(egn_link* link, const egn_opts* opts, double* eta_dev, double* pnli_dev);

/* Number of device and pinned-host allocations (cudaMalloc, cudaMallocHost) the
 * library has made in this process so far.  A diagnostic: it lets a caller check
 * that a sequence of calls (egn_nli_eta_static, for one) allocated nothing,
 * independently of other processes sharing the GPU. */
egn_status egn_allocation_count(long long* count);

/* ------------------------------------------------------------------ batches
 * Many links evaluated together (the paper evaluates one link at a time; its
 * parallel strategy distributes the islands of one link over workers).
 *
 * egn_batch_create snapshots n_links >= 1 links that have a comb
 * (egn_set_wdm) and share a device: each link's channel, segment and
 * Gauss-Legendre tables for `opts` are copied into batch-owned device memory,
 * so later egn_set_wdm calls or egn_link_destroy on the links do not affect
 * the batch.  It allocates one workspace per link and the outputs of all
 * links, runs the whole evaluation once (validation; egn_batch_read can read
 * its results), and captures it into a CUDA graph of every link's chain
 * (island planner, integrator passes, assembly): links too small to fill the
 * GPU are concurrent branches, links that fill it run one after the other.
 * opts->stream is ignored; opts->timeout_ms applies to egn_batch_read.
 * Errors as egn_nli_eta (the first failing link is reported).
 *
 * egn_batch_launch enqueues one evaluation of every link (one graph launch) on
 * `stream` (NULL = legacy default stream); asynchronous.  Launches on one
 * batch must not overlap on the GPU (they share the batch's workspaces).
 *
 * egn_batch_outputs gives the device arrays eta and P_NLI of all channels,
 * link after link, and the host array offsets[0..n_links] of each link's
 * first channel (offsets[n_links] = all channels); valid until destroy.
 *
 * egn_batch_read waits (opts->timeout_ms) for the work queued on `stream`,
 * checks every link's device status and copies eta and P_NLI of all channels
 * to host arrays of offsets[n_links] doubles (either may be NULL).
 *
 * egn_nli_eta_batch: one evaluation of n links without a graph; eta[i] and
 * pnli[i] are host arrays of link i's n_ch doubles (NULL entries skipped). */
typedef struct egn_batch egn_batch;
egn_status egn_batch_create(egn_link* const* links, int n_links, const egn_opts* opts, egn_batch** out);
egn_status egn_batch_launch(egn_batch* batch, void* stream);
egn_status egn_batch_outputs(const egn_batch* batch, const double** eta_dev, const double** pnli_dev,
                             const long long** offsets);
egn_status egn_batch_read(egn_batch* batch, void* stream, double* eta, double* pnli);
void egn_batch_destroy(egn_batch* batch);
egn_status egn_nli_eta_batch(egn_link* const* links, int n_links, const egn_opts* opts, double* const* eta,
                             double* const* pnli);

/* Per-island terms for parity checks on sampled islands: for each of n_isl
 * islands given as 4 ints (coi, n1, n2, n3), writes 5 doubles (D, E, F, G, H)
 * into terms_out (host), evaluated by the same device kernels as egn_nli_eta.
 * Terms whose Kronecker delta in Eq. 15 is zero are written as 0 unless
 * all_terms != 0.  A non-existent island yields zeros. */
egn_status egn_island_terms(egn_link* link, const egn_opts* opts, int n_isl, const int* coi_n1_n2_n3,
                            int all_terms, double* terms_out);

/* The island list of the current comb as planned on the device (for tests):
 * up to max entries of 4 ints (coi, n1, n2, n3) in the order the integrator
 * visits them (COI, then n1, n2, n3 ascending).  *count gets the total. */
egn_status egn_plan_islands(egn_link* link, long long max, int* coi_n1_n2_n3, long long* count);

/* Tuning of the kernels' launch shape (results do not change beyond rounding).
 *   EGN_TUNE_FP32C_POINTS_PER_THREAD: quadrature points per thread in the FP32C
 *   D/G/H pass, 4 (default: 64-thread CTAs, 10 per SM), 8 (128-thread CTAs, 3
 *   per SM) or 2 (128-thread CTAs, 8 per SM). */
enum { EGN_TUNE_FP32C_POINTS_PER_THREAD = 1 };
egn_status egn_set_tuning(egn_link* link, int param, int value);

/* Autotuning (Sec. III-D, Fig. 11: Delta z trades accuracy for time).  With
 * opts (segment form) as the base, evaluates the link at dz_ref_km, then the
 * n_candidates segment bounds dz_candidates from the coarsest down, and picks
 * the coarsest whose worst channel differs from the reference by at most
 * target_db (no candidate qualifies: dz_ref_km itself, error 0).  For
 * EGN_PREC_FP32C it then times 4 and 8 points per thread of the D/G/H pass at
 * the chosen Delta z (median of 5 device-timed evaluations each) and sets the
 * faster on the link (egn_set_tuning).  Synchronous; the link's own workspace
 * and a private stream are used.  Candidates finer than dz_ref_km are skipped. */
typedef struct {
    double dz_km;          /* chosen segment-length bound */
    int points_per_thread; /* FP32C D/G/H launch shape now set on the link */
    double max_err_db;     /* worst channel |10 log10(eta(dz) / eta(dz_ref))| */
    double ms;             /* device ms of one evaluation with the choice */
} egn_tune_result;
egn_status egn_autotune(egn_link* link, const egn_opts* opts, double target_db, const double* dz_candidates,
                        int n_candidates, double dz_ref_km, egn_tune_result* out);

/* Node rule of the island integrals (Eq. 17-21).
 *   EGN_RULE_GL     (default) the Gauss-Legendre panels of egn_opts.gl_order.
 *   EGN_RULE_RIDGE  a rule that resolves the ridges of |mu|^2 along f1 = f and
 *                   f2 = f (with chi of Eq. 5/24, |mu|^2 is close to a Lorentzian
 *                   in f1 - f of half-width alpha / (4 pi^2 |beta2 + 2 pi beta3 f|
 *                   |f2 - f|), far narrower than the channels): in each evaluation
 *                   order the outer range is cut at the knees of the outer
 *                   raised-cosine shape, wherever two inner break lines cross and
 *                   at a ridge of the outer variable; every inner interval at the
 *                   knees of the other two shapes and at the ridges inside it.  A
 *                   piece that ends on a ridge gets egn_opts.gl_order nodes graded
 *                   by x = x_r + h sinh(tau) (tau on a Gauss-Legendre rule, h the
 *                   ridge half-width; a piece with ridges at both ends is halved);
 *                   another piece gets max(n_min, ceil(gl_order x length /
 *                   interval)) Gauss-Legendre nodes.  The half-widths take the first
 *                   span's alpha, beta2 and beta3.  EGN_PREC_FP64 on any link;
 *                   EGN_PREC_FP32C on links of identical spans or of at most
 *                   four span types (graded nodes formed in FP32, within a few
 *                   1e-7 of their FP64 offsets from the ridge); gl_order <= 64
 *                   (other requests: EGN_E_UNSUPPORTED /
 *                   EGN_E_INVALID_ARG); egn_nli_eta_static refuses it; batches
 *                   take it through per-link passes (no flat work list).
 * The rule is a setting of the link; n_min is ignored for EGN_RULE_GL. */
enum { EGN_RULE_GL = 0, EGN_RULE_RIDGE = 1 };
egn_status egn_set_node_rule(egn_link* link, int rule, int n_min);

/* Choice of the node rule (Sec. III-D weighs accuracy against time; here the
 * quadrature of Eq. 17-21).  Evaluates the link -- in FP32C when opts asks for
 * it and the link has at most four span types, else in FP64 -- with the configured
 * Gauss-Legendre rule of opts->gl_order and with the ridge-resolving rule at
 * 4, 8, 16, ... nodes per piece, doubling until the worst channel moves by less
 * than target_db / 4 between two orders or max_nodes (4..64) is reached; that
 * last order stands for the converged value.  Picks the smallest order whose
 * worst channel lies within target_db of it, sets EGN_RULE_RIDGE (n_min 4) on
 * the link, and reports the chosen order, its error, the configured rule's
 * error against the same value and the device time of one evaluation at the
 * choice.  Synchronous; the caller evaluates with opts.gl_order = nodes in the
 * same precision.  On failure the link's node rule is left as it was. */
typedef struct {
    int rule;                 /* EGN_RULE_RIDGE */
    int nodes;                /* chosen nodes per piece */
    double max_err_db;        /* worst channel |10 log10(eta(nodes) / eta(reference))| */
    int reference_nodes;      /* the last order evaluated */
    double last_change_db;    /* worst channel change between the last two orders */
    double configured_err_db; /* the same error of the configured rule */
    double ms;                /* device ms of one evaluation with the choice */
} egn_rule_result;
egn_status egn_autotune_rule(egn_link* link, const egn_opts* opts, double target_db, int max_nodes,
                             egn_rule_result* out);

/* Per-stage device timing.  With profiling on, every evaluation records CUDA
 * events on its stream around five stages; egn_last_timings waits for the last
 * evaluation and writes up to max durations [ms] in the order: island planner,
 * D/G/H pass, E pass, F pass, assembly.  *n gets the number written. */
egn_status egn_set_profiling(egn_link* link, int enable);
egn_status egn_last_timings(egn_link* link, double* ms, int max, int* n);

/* EGN constants of a modulation format (EGN_FMT_*): Phi = mu4 - 2 and
 * Psi = mu6 - 9 mu4 + 12 with mu_k = E|a|^k / (E|a|^2)^(k/2) of the
 * equiprobable square QAM (0 for the Gaussian limit). */
egn_status egn_format_moments(int fmt, double* phi, double* psi);

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1] of order n (1..4096),
 * as used by the node rule; x and w hold n doubles each. */
egn_status egn_gauss_legendre(int n, double* x, double* w);

/* Thread-local message describing the last failure on this thread. */
const char* egn_last_error(void);

/* Library version string. */
const char* egn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EGN_H */
