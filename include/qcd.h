/*
 * qcd.h - C ABI of the GB300 nested-BiCGStab / SAP / ll-SSOR solver for the
 * clover-preconditioned O(a)-improved Wilson-Dirac equation
 *
 *     D x = b,   D = 1 - kappa F H                                   (Eq. (1), Eq. (2))
 *
 * of T. Boku, K.-I. Ishikawa et al., "Multi-block/multi-core SSOR
 * preconditioner for the QCD quark solver for K computer", Lattice 2012.
 *
 * H is the 8-neighbour hop with SU(3) links and (1 -/+ gamma_mu) spin
 * projectors, F(n) the inverse clover term (Eq. (2) and the sentence after
 * it).  The solver is the paper's nested BiCGStab (Sec. 2): an FP64 outer
 * flexible BiCGStab whose preconditioner is an FP32 inner BiCGStab, right-
 * preconditioned by Luescher's SAP, M_SAP = K sum_{j<N_SAP} (1 - D K)^j
 * (Eq. (4), Alg. 1), whose block inverses A_EE / A_OO are SSOR sweeps in
 * locally-lexicographic sub-block order (Sec. 3, "Inverse of block operator").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - dims = {Lx, Ly, Lz, Lt}; site n = x + Lx*(y + Ly*(z + Lz*t)).
 *    mu = 0..3 is x, y, z, t (the paper's mu = 1..4, mu = 4 the time axis).
 *  - Complex numbers are interleaved (re, im).  Canonical caller layouts:
 *      links   U[n][mu][a][b]          complex128 (4 x 3 x 3 complex per site)
 *      spinor  psi[rhs][n][spin][colour] complex128 (FP64) or complex64 (FP32)
 *  - gamma matrices in the Dirac representation with gamma_4 diagonal
 *    (Sec. 3, "Dirac representation"): gamma_k = [[0,-i s_k],[i s_k,0]],
 *    gamma_4 = diag(1,1,-1,-1).  The basis is part of the ABI.
 *  - Boundary conditions periodic; qcd_set_boundary(ctx, -1) makes the
 *    fermion hops across the t edge antiperiodic.
 *  - SAP blocks: block[mu] divides L_mu and L_mu/block[mu] is even and >= 2
 *    (so the block checkerboard of Eq. (3) is consistent); subblock[mu]
 *    divides block[mu].  Block colour = (sum_mu floor(n_mu/block_mu)) mod 2,
 *    colour 0 is E.
 *
 * Ownership and streams
 * ---------------------
 *  - A context owns its copies of the links, the clover field and all work
 *    vectors (device memory it allocates with cudaMalloc and frees in
 *    qcd_destroy).  The caller owns every pointer it passes.
 *  - Spinor pointers may be device pointers or host pointers (pageable or
 *    pinned); host data is copied in and out inside the call on the context
 *    stream.  Device pointers must stay valid until the work completes.
 *  - All device work is enqueued on the stream given to qcd_create (NULL =
 *    legacy default stream).  qcd_apply_D and qcd_sap_precondition with
 *    device pointers are asynchronous; every call with host pointers, and
 *    qcd_solve, synchronise the stream before returning.
 *  - One context per host thread.
 *
 * Errors
 * ------
 *  Calls return QCD_OK or a negative status and never abort, exit or trap.
 *  qcd_last_error gives a message.  A CUDA error poisons the context: every
 *  later call returns QCD_ERR_STATE.
 */
#ifndef QCD_H
#define QCD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qcd_ctx qcd_ctx;

enum {
    QCD_OK = 0,
    QCD_ERR_ARG = -1,       /* invalid argument (sizes, geometry, parameters)          */
    QCD_ERR_CUDA = -2,      /* a CUDA runtime call failed; the context is poisoned    */
    QCD_ERR_OOM = -3,       /* device allocation failed                               */
    QCD_ERR_SINGULAR = -4,  /* a chiral 6x6 block of the clover term is not invertible */
    QCD_ERR_NOCONV = -5,    /* max_outer reached (x holds the last iterate), or a
                               right-hand side holds a non-finite value (that one is
                               not iterated; the others are solved as usual)        */
    QCD_ERR_BREAKDOWN = -6, /* BiCGStab breakdown not cured by 5 restarts             */
    QCD_ERR_TIMEOUT = -7,   /* a bounded device-side wait gave up                     */
    QCD_ERR_STATE = -8      /* wrong call order, or context poisoned by a CUDA error  */
};

/* Precisions and storage forms.  QCD_F16 is the half-precision storage of the precision
 * pattern (FP32 arithmetic); the value 3 is not used (the SAP block spinors are kept per block in
 * units of their largest source component, so FP16's 10-bit mantissa, not BF16's exponent
 * range, is what the storage needs).  QCD_F32X2 is pair-of-FP32 arithmetic: each FP64 link and
 * clover entry held as hi + lo FP32 numbers, products and sums carried without losing the low
 * part (Dekker's product with the FMA error term, Knuth's TwoSum), on an FP32 input; about 2^-46
 * relative per site, on the FP32 pipe. */
enum { QCD_F64 = 0, QCD_F32 = 1, QCD_F16 = 2, QCD_F32_SU3 = 4, QCD_F32X2 = 5 };

/* Solver and SAP parameters (Sec. 2, Sec. 3, Eq. (4)). */
typedef struct {
    double kappa, csw;  /* must equal the values given to qcd_build_clover             */
    int block[4];       /* SAP block extents (x, y, z, t)                              */
    int subblock[4];    /* ll-ordering sub-block extents; subblock | block             */
    double omega;       /* SSOR relaxation, 0 < omega < 2                              */
    int nsweep;         /* SSOR sweeps (forward + backward pass) per block inverse, or
                           minimal-residual steps when block_solver = 1                */
    int nsap;           /* SAP cycles N_SAP                                            */
    double tol;         /* outer: stop at ||b - D x|| <= tol ||b|| (true FP64 residual) */
    double inner_tol;   /* inner: stop at ||r|| <= inner_tol ||q||                     */
    int max_outer, max_inner;
    int bc_t;           /* +1 periodic, -1 antiperiodic in t (must match qcd_set_boundary) */
    int sap_storage;    /* QCD_F32 (plain) or QCD_F16 (half storage, FP32 arithmetic)    */
    int learned;        /* 0: plain SAP.  1: precondition with M_SAP + N (1 - D M_SAP),
                           N the learned correction (qcd_learned_*), unless the last
                           qcd_learned_evaluate found it slower than plain SAP, in
                           which case plain SAP is used (the fallback).  2: always use
                           the learned correction                                     */
    int sap_ctas;       /* SSOR kernel form, as qcd_set_sap_ctas (-1..16); 0 = context
                           setting; results do not depend on it                       */
    int block_solver;   /* SAP block inverse A_BB.  0: ll-ordered SSOR (Sec. 3; uses
                           subblock, omega, nsweep).  1: the even-odd alternative
                           Sec. 3 compares it with: nsweep minimal-residual steps on
                           the Schur complement 1 - kappa^2 F_e H_eo F_o H_oe of each
                           block's even sites from 0, then the odd sites
                           (sap_storage QCD_F32 and learned 0 only; subblock must
                           still divide block; omega unused)                         */
    int rhs_group;      /* qcd_solve: right-hand sides solved together (the batched
                           iteration); more are solved group after group, each in the
                           device memory of one group.  0: as many as fit the free device
                           memory (at least 1).  Results do not depend on it: each
                           right-hand side's iterates are those of its solve alone      */
    int outer_precision; /* qcd_solve, the outer BiCGStab's v = D p^ and t = D s^ (Sec. 2):
                           QCD_F64 (0, the default): the FP64 D.  QCD_F32X2: the
                           pair-of-FP32 D of the inner solver's FP32 output (exact in FP32),
                           within about 1e-13 of the FP64 D and several times faster on
                           GB300, whose FP64 rate is 1/64 of its FP32 rate.  QCD_F32: the FP32 D
                           applied to the inner solver's FP32 solution, widened to FP64;
                           FP64 then serves only the true residual b - D x, the dot
                           products and norms, and x.  The recursive residual then
                           carries the FP32 error of D, so reaching tol takes restarts
                           from the true residual                                     */
} qcd_params;

typedef struct {
    int status;
    int outer_iters;     /* outer iterations (summed over right-hand-side groups)       */
    int inner_iters;     /* inner iterations summed over the right-hand sides           */
    int restarts;        /* restarts from the true residual, summed over them           */
    double true_rel_res; /* max over right-hand sides of ||b - D x|| / ||b|| (FP64)     */
    double ms_total;     /* wall time of the call                                      */
    double ms_dslash;    /* device ms of the D kernels (FP32 and FP64) during the call
                            when kernel profiling is on (qcd_set_profiling), else 0     */
    double ms_sap;       /* the same for the SAP kernels (block solves, hop updates)    */
} qcd_stats;

/* Creates a context for a lattice of the given extents (each >= 2, even
 * volume).  cuda_stream is a cudaStream_t (NULL = default stream).  The
 * current CUDA device at this call is the context's device. */
int qcd_create(qcd_ctx **ctx, const int dims[4], void *cuda_stream);
void qcd_destroy(qcd_ctx *ctx);
const char *qcd_last_error(const qcd_ctx *ctx);

/* Fermion boundary condition in t: +1 periodic (default), -1 antiperiodic. */
int qcd_set_boundary(qcd_ctx *ctx, int bc_t);

/* Copies the links U (canonical complex128 [V][4][3][3]; host memory if
 * on_device == 0, device memory otherwise) into the context's internal FP64
 * and FP32 link fields (Eq. (2): U_mu(n)).  Invalidates the clover field. */
int qcd_load_gauge(qcd_ctx *ctx, const double *U, int on_device);

/* Builds F(n) = (1 - (c_SW kappa/2) sigma_{mu nu} F_{mu nu}(n))^{-1} (Eq. (2)),
 * F_{mu nu} the clover-leaf field strength (Q - Q^dag)/(8i) of the loaded
 * links, in FP64 and inverts it per chiral 6x6 block (Sec. 3: the clover term
 * is stored in the chiral representation).  Requires qcd_load_gauge.
 * Returns QCD_ERR_SINGULAR if some block has a pivot below 1e-300. */
int qcd_build_clover(qcd_ctx *ctx, double kappa, double csw);

/* out = D in for nrhs right-hand sides (Eq. (2)).  prec = QCD_F64: in/out are
 * complex128 [nrhs][V][4][3]; QCD_F32: complex64; QCD_F16: complex64 in/out
 * with the links and the clover field stored in FP16 (FP32 arithmetic; the
 * FP16 copies are made on first use after each field change); QCD_F32_SU3:
 * complex64 in/out with each link stored as its first two rows and the third
 * rebuilt as the conjugate cross product (SU(3) 12-real form, Table 1: 672
 * instead of 768 bytes per site); QCD_F32X2: complex64 in, complex128 out, computed in
 * pair-of-FP32 arithmetic from the FP64 fields (hi + lo copies made on first use after each
 * field change), within about 1e-13 of the FP64 D of the same input.  in and out must not
 * overlap.  Requires qcd_build_clover. */
int qcd_apply_D(qcd_ctx *ctx, void *out, const void *in, int prec, int nrhs);

/* out = M_SAP in (Eq. (4), Alg. 1) in FP32 for nrhs right-hand sides:
 * complex64 [nrhs][V][4][3].  Uses p->block, p->subblock, p->omega,
 * p->nsweep, p->nsap, p->sap_storage.  All right-hand sides go through one
 * batched application (one grid row of block solves per right-hand side);
 * each result equals, bit for bit, the call with that one alone.  Device
 * scratch grows to 4 nrhs + 1 complex64 fields (7 nrhs + 1 with
 * p->block_solver = 1). */
int qcd_sap_precondition(qcd_ctx *ctx, float *out, const float *in, const qcd_params *p, int nrhs);

/* The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory at call time: a process whose framework
 * allocator has already reserved the GPU's free memory (a cudaMalloc here
 * would fail or fragment its pool), or a serving loop with a fixed memory
 * budget that must not grow or stall on an allocation while work is in
 * flight.  Such a caller creates the context, loads the gauge field and
 * builds the clover term once at set-up (those calls allocate), then calls
 * this instead of qcd_sap_precondition.
 *
 * out = M_SAP in, exactly as qcd_sap_precondition with nrhs = 1, for device
 * pointers only (16-byte aligned complex64 [V][4][3]), with
 * p->sap_storage = QCD_F32, p->learned = 0 and p->block_solver = 0 (others
 * are rejected with QCD_ERR_ARG); p->sap_ctas (-2..16, 0 = the context's
 * qcd_set_sap_ctas setting) picks the SSOR kernel form as for
 * qcd_sap_precondition.  It calls no cudaMalloc, cudaFree or allocating
 * library routine: its scratch (four FP32 spinor fields, the per-site SSOR
 * records and the ll-schedule tables) is one fixed __device__ array of about
 * 68.3 MB that every GPU loading the library holds until the process exits.
 * Lattices above 41,472 sites (12^3 x 24) are rejected with QCD_ERR_ARG.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * The array keeps the schedule tables and records of the last call (per
 * device): a call with the same context, unchanged fields, geometry and form
 * only launches kernels and is asynchronous on the context stream; any other
 * call first rebuilds them, which copies from host memory and synchronises the
 * context stream (so it cannot be captured either).  All calls on a device
 * share the one array and leave their data in it; every region is rewritten
 * before it is read, but calls that overlap on the GPU (other streams, other
 * contexts on the same device) race and must be serialised by the caller. */
int qcd_sap_precondition_noalloc(qcd_ctx *ctx, float *out, const float *in, const qcd_params *p);

/* Solves D x = b (Eq. (1)) by the nested BiCGStab of Sec. 2 for nrhs
 * right-hand sides (complex128 [nrhs][V][4][3]), all advancing together
 * (batched kernels, per right-hand side scalars on the device; a converged
 * right-hand side drops out).  x holds the initial guess
 * on entry (zero it for x0 = 0) and the solution on return.  Synchronises.
 * st may be NULL.  Returns QCD_OK when every right-hand side reached the
 * true relative residual p->tol. */
int qcd_solve(qcd_ctx *ctx, double *x, const double *b, const qcd_params *p, int nrhs,
              qcd_stats *st);

/* Solves n independent problems at once: instance i is ctxs[i] (its own
 * lattice, gauge field, clover field and kappa) with x[i], b[i], params[i],
 * nrhs[i] as in qcd_solve.  The instances run concurrently on the GPU, each on
 * its context's stream driven by its own host thread, so that small lattices
 * fill the SMs a large one leaves idle.  Every context must have its own
 * stream, other than the legacy default stream (QCD_ERR_ARG otherwise), and
 * none may be used by another thread during the call.  stats (may be NULL):
 * [n], one per instance.  Returns the first non-OK status in instance order,
 * QCD_OK when all converged.  No counterpart in the paper. */
int qcd_solve_multi(int n, qcd_ctx *const *ctxs, double *const *x, const double *const *b, const qcd_params *params,
                    const int *nrhs, qcd_stats *stats);

/* on != 0 (default): when the context stream is not the legacy default stream
 * and kernel profiling is off, qcd_solve captures each inner BiCGStab solve as
 * one CUDA graph: a conditional while node repeats the inner iteration until a
 * kernel finds no right-hand side active or max_inner reached, so convergence
 * is decided on the device and the host waits once per inner solve (where the
 * driver has no conditional nodes, one iteration is captured and replayed, the
 * host reading the active flags after each).  Results do not depend on it. */
int qcd_set_graphs(qcd_ctx *ctx, int on);

/* Tuning knob of the SAP block kernel; results do not depend on it.  The
 * block solve has two forms.  The warp form runs 32 lanes (or 8, see
 * qcd_set_sap_form) per site update over
 * a cluster of C CTAs per block (C <= 16, each CTA owning an equal share of
 * every dependency level of the sweep and keeping its sites' spinors in its
 * shared memory, which must fit).  The thread form (FP32 storage, blocks whose
 * spinor fits one CTA) runs one thread per site update with the block's links
 * and clover field stored per block in level order.  min_ctas >= 1: the warp
 * form with the smallest such C >= min_ctas.  0 (default): the warp form with
 * the largest C in {1, 2, 4, 8} for which one colour's clusters still fit the
 * SM count (at least the smallest C that fits).  -1: the thread form where it
 * fits, else as 0.  More CTAs per block spread a level's sites over more SMs
 * at the price of more cluster barriers. */
int qcd_set_sap_ctas(qcd_ctx *ctx, int min_ctas);

/* Second tuning knob of the warp form above: lanes per site update.  form = 1:
 * 32 lanes (lane = hop direction and colour row, one update per warp); 2: 8
 * lanes (lane = hop direction, four updates per warp: about two thirds of the
 * issued instructions, but a quarter of the warps to hide latency); 0 (default):
 * per launch, the 8-lane form where the grid keeps at least 16 of its warps
 * resident per SM (many small blocks, several right-hand sides), else 32.
 * Both perform the same rounding steps in the same order: results are
 * identical bit for bit.  QCD_ERR_ARG outside 0..2. */
int qcd_set_sap_form(qcd_ctx *ctx, int form);

/* Diagnostic, host only (needs no GPU and no context): the schedule of the
 * SSOR block kernel that a context with these lattice extents would run for
 * SAP blocks `block` with ll sub-blocks `subblock` (Sec. 3), sap_ctas as in
 * qcd_set_sap_ctas, half = 1 for FP16 storage, planned for an SM count `sms`
 * (the automatic cluster width depends on it; GB300: 152).  Every site of a
 * block has a dependency level (a site's level is one more than the highest
 * level of its in-block neighbours earlier in the ll order); each CTA of the
 * block's cluster owns some sites of every level; each level is cut into
 * chunks (timeline steps of the forward pass; the backward pass runs them in
 * reverse, step 2 nchunks - 1 - c for chunk c), and a barrier flag before a
 * step orders the steps that exchange data (1: CTA barrier, 2: cluster
 * barrier).  meta[8] receives: sites per block, levels, CTAs per block (C),
 * chunks, most sites of one CTA in one chunk, most sites one CTA owns,
 * thread form (0/1), shared memory bytes per CTA.  The arrays, each NULL or
 * sized as stated, receive per block-local site (lexicographic, x fastest;
 * meta[0] entries): its level, its owning CTA, its offset in that CTA's slab
 * of the block spinor, its chunk; and flags[2 * meta[3]] per timeline step.
 * Call with NULL arrays first to learn the sizes.  QCD_ERR_ARG for a
 * geometry the library rejects. */
int qcd_sap_plan_tables(const int dims[4], const int block[4], const int subblock[4], int sap_ctas, int half,
                        int sms, int meta[8], int *level, int *owner, int *slot, int *chunk,
                        unsigned char *flags);

/* Autotuner (no counterpart in the paper, which fixes 6^4 blocks with 3^4
 * sub-blocks).  Starting from *base (kappa, csw, tol, inner_tol, bc_t, limits),
 * times complete solves of D x = b from x0 = 0 for candidate SAP set-ups and
 * returns the fastest that converges in *best (block, subblock, omega,
 * sap_storage, sap_ctas, nsweep, nsap, outer_precision, rhs_group) and its time
 * in *best_ms.  Stage 1
 * tries block extents (2, 3, 4, 6, 8, 12 or 16, the spatial ones alike, the
 * time extent one to two times the spatial one, each dividing L with an even
 * quotient) with sub-blocks block/2, block/3 or block, blocks of about 256 sites
 * first, each with FP16 storage and the tile form (sap_ctas -2; the cluster form
 * where the block does not fit), 2 sweeps, 2 cycles and omega 1; stage 2 is a
 * coordinate search from the fastest, keeping each move that is faster: the
 * outer operator in pair-of-FP32 arithmetic (outer_precision QCD_F32X2, the same
 * accuracy) where base asks for QCD_F64, omega upwards in steps of 0.2 while it
 * improves, nsap 1 or 3, nsweep 3 or 1, then the storage and kernel forms
 * (FP32 / FP16, sap_ctas -2, 0, 2).  At most
 * max_candidates solves are timed (<= 0: 64), at most half of them in stage 1.
 * Stage 3 (nrhs > 1 and base->rhs_group = 0) then times the winner with
 * right-hand sides in groups of 1, 2, 4 or 8 dividing nrhs, as well as all at
 * once, and keeps the fastest rhs_group.
 * b: complex128 [nrhs][V][4][3], host or device.  Synchronises. */
int qcd_autotune(qcd_ctx *ctx, const double *b, int nrhs, const qcd_params *base, qcd_params *best,
                 double *best_ms, int max_candidates);

/* Tuning cache (no counterpart in the paper): with a path set, qcd_autotune first looks for a
 * result stored under the same key (lattice extents, nrhs, kappa, csw, bc_t, tolerances and
 * limits, omega, rhs_group, max_candidates, GPU name and SM count, tuner version) and returns it
 * without timing anything; otherwise it tunes and appends the winner as one JSON object per
 * line ({"key": ..., "block": [...], "subblock": [...], "omega", "sap_storage", "sap_ctas",
 * "nsweep", "nsap", "rhs_group", "outer_precision", "ms"}).  NULL or "" switches the cache off (the default).  Process-wide;
 * the file is read and appended under a lock.  Always QCD_OK. */
int qcd_set_tune_cache(const char *path);

/* ---- learned correction (no counterpart in the paper) -----------------------
 * N is a linear, gauge-covariant network of 3 parallel-transport layers with
 * 1 -> 8 -> 8 -> 1 channels: y_c(n) = sum_{d=0..8} sum_{c'} W_d[c][c'] (T_d x_c')(n),
 * T_0 = 1, T_{2mu+1} x(n) = U_mu(n) x(n+mu), T_{2mu+2} x(n) = U_mu(n-mu)^dag x(n-mu)
 * (the directions 1..8 are (mu, forward/backward)), W_d[c][c'] a 4x4 complex
 * spin matrix.  Weights: complex64 [layer][9][cout][cin][4][4], concatenated.
 * Layers run on the tensor cores in BF16 with FP32 accumulation.  Because N is
 * linear, M_SAP + N (1 - D M_SAP) is a fixed preconditioner for the inner
 * BiCGStab (qcd_params.learned = 1). */
long qcd_learned_weight_count(void);
/* w: complex64 [n], host or device; resets the optimiser state */
int qcd_learned_set_weights(qcd_ctx *ctx, const float *w, long n);
/* w: host complex64 [n] */
int qcd_learned_get_weights(qcd_ctx *ctx, float *w, long n);
/* Weights file of the correction: one JSON header line ({"format": "qcd-learned-weights",
 * "version": 1, "layers", "channels", "layout", "dtype": "complex64", "count"}) followed by the
 * count complex64 weights in the layout above.  qcd_learned_save writes the current weights
 * (QCD_ERR_STATE without any); qcd_learned_load reads them and sets them as
 * qcd_learned_set_weights does, and rejects a file whose header or size does not match this
 * network with QCD_ERR_ARG.  Synchronise. */
int qcd_learned_save(const qcd_ctx *ctx, const char *path);
int qcd_learned_load(qcd_ctx *ctx, const char *path);
/* out = N(in), complex64 [V][4][3], host or device */
int qcd_learned_apply(qcd_ctx *ctx, float *out, const float *in);
/* One training pair: loss = |N(rho) - eps|^2 / |eps|^2 and its gradient grad
 * (host float [2n]: 2 (Re, Im) of dL/dW* per complex weight).  rho, eps:
 * complex64 [V][4][3], host or device. */
int qcd_learned_loss_grad(qcd_ctx *ctx, const float *rho, const float *eps, double *loss, float *grad);
/* Trains N on npairs pairs made from the sources r_k (complex64
 * [npairs][V][4][3], host or device) with the plain SAP of *p:
 * rho_k = r_k - D M_SAP r_k, eps_k = D^{-1} rho_k (the error of M_SAP r_k,
 * solved in FP64 to 1e-9), loss sum_k |N(rho_k) - eps_k|^2 / |eps_k|^2, Adam
 * with learning rate lr over mini-batches of `batch` pairs for `epochs`
 * epochs.  history (may be NULL): [epochs + 1] mean loss before training and
 * after each epoch.  Requires qcd_learned_set_weights (the initial weights). */
int qcd_learned_train(qcd_ctx *ctx, const float *sources, int npairs, const qcd_params *p, int epochs, int batch,
                      float lr, double *history);

/* Result of qcd_learned_evaluate: the same right-hand sides solved from x = 0
 * with plain SAP and with the learned correction (times are wall times of a
 * second, warm qcd_solve call; relres the FP64 true relative residual). */
typedef struct {
    double plain_ms, learned_ms;
    double plain_relres, learned_relres;
    int plain_outer, plain_inner;
    int learned_outer, learned_inner;
    int use_learned; /* 1: learned converged and was faster; qcd_params.learned = 1 uses it */
    int pad;
} qcd_learned_verdict;

/* Assesses the trained correction on b (complex128 [nrhs][V][4][3], host or
 * device) with the solver settings *p (p->learned ignored): solves with plain
 * SAP and with the correction, compares time to solution, and records the
 * verdict in the context; qcd_learned_set_weights and qcd_learned_train clear
 * it.  Synchronises. */
int qcd_learned_evaluate(qcd_ctx *ctx, const double *b, int nrhs, const qcd_params *p, qcd_learned_verdict *out);

/* ---- measurement hooks -------------------------------------------------- */

/* Kernel classes timed when profiling is on. */
enum {
    QCD_K_DSLASH32 = 0, /* full operator D in FP32 (inner solver)     */
    QCD_K_DSLASH64 = 1, /* full operator D of the outer solver: FP64,
                           or pair-of-FP32 arithmetic (QCD_F32X2)     */
    QCD_K_SSOR = 2,     /* SAP block SSOR (A_EE / A_OO)              */
    QCD_K_SAPHOP = 3,   /* SAP block / cross-block hop updates       */
    QCD_K_BLAS = 4,     /* BiCGStab vector updates and reductions    */
    QCD_K_OTHER = 5,    /* layout conversion, clover build           */
    QCD_K_LEARNED = 6,  /* learned correction (layers, gradients)    */
    QCD_K_COUNT = 7
};

/* on != 0: bracket every kernel launch with CUDA events on the context
 * stream and accumulate per-class device time. */
int qcd_set_profiling(qcd_ctx *ctx, int on);
/* Launch count and device milliseconds per class since the last reset
 * (synchronises the stream).  reset != 0 clears the counters afterwards. */
int qcd_kernel_stats(qcd_ctx *ctx, int kclass, long *launches, double *ms, int reset);
/* Total kernel launches made by this context since creation. */
long qcd_launch_count(const qcd_ctx *ctx);

/* Test hook: the next `count` outer BiCGStab iterations of qcd_solve start from rho = 0 for
 * every active right-hand side, the state a vanishing <rhat, r> leaves (a breakdown made on the
 * host; no device fault is involved).  The solver then takes its breakdown path: true residual,
 * restart from it, and QCD_ERR_BREAKDOWN after 5 restarts of a right-hand side.  0 disarms. */
int qcd_debug_inject_breakdown(qcd_ctx *ctx, int count);

/* Test hook of the tensor-core learned layer: with on != 0 its kernel issues no MMA and commits
 * nothing to its mbarriers, so its first wait for a commit finds none.  Every such wait is
 * bounded (about a second); the kernel stops, frees its tensor memory and returns, and the call
 * that launched it reports QCD_ERR_TIMEOUT, leaving the context usable.  The failure path is
 * exercised without a device fault.  0 disarms. */
int qcd_debug_tc_skip_commit(qcd_ctx *ctx, int on);

/* D on internal-layout buffers only, repeated `iters` times (no layout
 * conversion): the kernel the memory-bandwidth roofline is measured on.
 * prec = QCD_F64, QCD_F32, QCD_F16, QCD_F32_SU3 or QCD_F32X2; nrhs >= 1.  Work buffers are
 * allocated on first use and kept. */
int qcd_bench_dslash(qcd_ctx *ctx, int prec, int nrhs, int iters);

/* Measured FP32 FMA throughput of the context's GPU in TFLOP/s (2 flop per FMA): independent
 * FMA chains in registers over every SM, iters x 4096 FMAs per thread, timed with CUDA events on
 * the context stream.  The denominator of the SAP block kernel's arithmetic roofline.
 * Synchronises. */
int qcd_bench_fp32_peak(qcd_ctx *ctx, int iters, double *tflops);

/* Measures the shared-memory load bandwidth of the GPU (GB/s, all SMs): conflict-free 16-byte
 * loads from a 32 KB buffer, four CTAs of 512 threads per SM; iters scales the run time
 * (64 is about a millisecond).  Synchronises. */
int qcd_bench_smem_peak(qcd_ctx *ctx, int iters, double *gbs);

#ifdef __cplusplus
}
#endif
#endif /* QCD_H */
