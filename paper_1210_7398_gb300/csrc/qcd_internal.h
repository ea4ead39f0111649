// Internal declarations of the GB300 solver library (not part of the C ABI).
//
// Internal field layouts (all in device memory, V sites, site order as the
// canonical lexicographic order n = x + Lx*(y + Ly*(z + Lz*t))):
//   FP64 spinor   [nrhs][12][V] double2   plane k = spin*3 + colour
//   FP32 spinor   [nrhs][6][V]  float4    plane p holds components 2p, 2p+1
//   FP64 links    [4][9][V]     double2   plane mu*9 + a*3 + b
//   FP32 links    [4][9][V]     float2
//   FP64 clover   [36][V]       double2   chiral blocks of F/2, packed (see clover.cu)
//   FP32 clover   [18][V]       float4    the same 72 reals per site
// Each plane is contiguous over sites, so a warp of consecutive sites reads
// one contiguous segment per plane (coalesced 16-byte or 8-byte loads).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qcd.h"

namespace qcd {

struct Lattice {
    int L[4];
    long V;
};

// SAP geometry: block decomposition (Eq. (3)) plus the ll-order schedule of
// the SSOR passes, grouped into dependency levels (steps) whose sites are
// pairwise non-adjacent.  For the SSOR kernel each block is dealt over C CTAs
// (a thread-block cluster when C > 1), each CTA owning an equal share of every
// level, and each level into chunks of at most nslot sites per CTA; the chunks
// form the kernel's timeline (forward pass, then the reversed backward pass).
// flags[p] (p < 2*nchunks) asks for a CTA (1) or cluster (2) barrier before
// timeline step p of every sweep.
struct SapPlan {
    int b[4] = {0, 0, 0, 0}, s[4] = {0, 0, 0, 0};
    int nb[4] = {0, 0, 0, 0};
    int vol = 0;        // sites per block
    int nsteps = 0;     // parallel steps per pass
    int max_step = 0;   // largest number of sites in one step
    int nblk[2] = {0, 0};
    std::vector<int> h_step_ptr, h_step_site, h_origin[2];
    int *d_origin[2] = {nullptr, nullptr};  // [nblk[c]][4] block origins per colour
    bool half = false;  // FP16 storage of the block spinor and the records (FP32 arithmetic)
    bool thread = false;  // thread form of the SSOR kernel (SoA per-block fields instead of records)
    bool tile = false;    // right-hand-side tiled thread form (ssor_tile.cu): per-block records in level order
    int C = 1, slab_vol = 0;  // CTAs per block (cluster), most sites one CTA owns
    int nchunks = 0, nslot = 0, nwarps = 0;
    int sms = 1;        // SM count of the device the plan was made for
    size_t smem_bytes = 0;
    std::vector<int> h_chunk_ptr;   // [C][nchunks + 1], offsets into h_chunk_site
    std::vector<int> h_chunk_site;  // block-local site indices, CTA-major
    std::vector<unsigned char> h_flags;  // [2 * nchunks]
    std::vector<int> h_site_off;    // [vol] global index offset of a block-local site from its block origin
    std::vector<int> h_own;         // [vol] (owning CTA << 24) | index in that CTA's slab of y
    std::vector<int> h_own_off;     // [C][slab_vol] global offset of each owned site, -1 past the last
    std::vector<int> h_pos;         // thread form: [vol] level position of each block-local site
    std::vector<int> h_origin_site[2];  // [nblk[c]] global index of each block origin
    int *d_chunk_ptr = nullptr;
    int2 *d_chunk_site = nullptr;   // (block-local site, global offset from the block origin)
    unsigned char *d_flags = nullptr;
    int *d_site_off = nullptr;
    int *d_own = nullptr;
    int *d_own_off = nullptr;
    int *d_pos = nullptr;
    int *d_origin_site[2] = {nullptr, nullptr};
    std::vector<int4> h_tile_pos;   // tile form: [vol][2] per level position (offset, slots, site)
    int4 *d_tile_pos = nullptr;
    int *d_lev_ptr = nullptr;       // tile form: [nsteps + 1] level boundaries (h_step_ptr)
    int tile_zslots = 1;            // tile form: zero slots after the vol site slots
    float *d_rec = nullptr;         // per-site records (links, clover, neighbour codes), V x 912 bytes
    long rec_version = -1;          // field version the records were built from
};

// learned correction: channels 1 -> 8 -> 8 -> 1, weights complex [9][cout][cin][4][4] per layer
constexpr int kLearnedLayers = 3;
constexpr int kLearnedChans[kLearnedLayers + 1] = {1, 8, 8, 1};

struct Learned {
    bool ready = false;
    int verdict = -1;        // last qcd_learned_evaluate: -1 none, 0 plain SAP faster, 1 learned faster
    long step = 0;           // Adam steps taken
    float2 *W = nullptr;     // FP32 master weights (complex)
    float2 *grad = nullptr;  // accumulated gradient, real pairs 2 (Re, Im) of dL/dW*
    float2 *m = nullptr, *v = nullptr;  // Adam moments
    __nv_bfloat16 *B = nullptr;  // BF16 real-block weight matrices, forward and adjoint per layer
    float *P = nullptr;      // weight-gradient accumulator of one layer [9][64][64]
    double *scal = nullptr;  // loss, |eps|^2
    long V = 0;              // lattice the activations are sized for
    void *act = nullptr;     // one allocation for the buffers below
    void *a1 = nullptr, *a2 = nullptr;   // hidden activations (BF16, 8 channels)
    float2 *g1 = nullptr, *g2 = nullptr, *g3 = nullptr, *tmp = nullptr;
    float4 *pairs = nullptr;  // training pairs: rho (plane FP32) then eps (site FP32) per pair
    size_t pairs_bytes = 0;
};

struct Profiler {
    bool on = false;
    long launches[QCD_K_COUNT] = {};
    double ms[QCD_K_COUNT] = {};
    struct Pending { int kclass; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
};

}  // namespace qcd

struct qcd_ctx {
    long uid = 0;        // unique per context of the process (never reused)
    int device = 0;
    cudaStream_t stream = nullptr;
    qcd::Lattice lat{};
    int bc_t = 1;
    std::string err;
    bool poisoned = false;
    long total_launches = 0;
    long graph_launches = 0;  // kernel launches inside one replay of the captured inner iteration
    qcd::Profiler prof;

    // gauge and clover fields
    bool have_gauge = false, have_clover = false;
    double kappa = 0, csw = 0;
    double2 *U64 = nullptr;
    float2 *U32 = nullptr;
    double2 *F64 = nullptr;
    float4 *F32 = nullptr;
    __half2 *U16 = nullptr;  // FP16 copies for the FP16-storage operator, made on first use
    uint2 *F16 = nullptr;    // [18][V], four halves per plane
    long half_version = -1;  // field_version the FP16 copies were made from
    float4 *U12 = nullptr;   // links as their first two rows [4][3][V] (SU(3) 12-real form), made on first use
    long u12_version = -1;
    float4 *Ux2 = nullptr;   // links [4][9][V] and clover [36][V] as hi + lo FP32 pairs (pair-arithmetic D)
    float4 *Fx2 = nullptr;
    long x2_version = -1;
    int *d_status = nullptr;  // device status word (clover singularity)

    // SAP plan cache (one geometry at a time)
    qcd::SapPlan plan;
    // learned correction
    qcd::Learned net;
    long field_version = 0;  // bumped whenever the links or the clover field change
    int sap_min_ctas = 0;    // lower bound on the CTAs (cluster size) per SAP block; 0: fill the SMs
    int sap_ctas_user = 0;   // the qcd_set_sap_ctas setting, which params with sap_ctas = 0 use
    int sms_override = 0;    // SM count the SAP plan is made for (0: ask the device); diagnostics
    int sap_form = 0;        // SSOR lanes per site update: 0 by occupancy, 1 warp form (32), 2 octet form (8)
    int inject_breakdown = 0;  // test hook: outer iterations still to start from rho = 0 (a host-made breakdown)
    bool tc_skip_commit = false;  // test hook: the tensor-core layer issues no MMA or commit (its waits run out)

    // workspace, grown on demand
    std::vector<void *> allocations;
    void *ws64 = nullptr;
    size_t ws64_bytes = 0;
    void *ws32 = nullptr;
    size_t ws32_bytes = 0;
    double *d_red = nullptr;      // reduction partials [nrhs][3][kRedMaxBlocks]
    double *d_red_tiles = nullptr;  // per-CTA partials of the fused D [nrhs][3][V / 128]
    double *d_scalars = nullptr;  // reduction results [nrhs][3]
    double *h_scalars = nullptr;  // pinned host mirror
    int red_rhs = 0;              // right-hand sides d_red / d_scalars are sized for
    void *d_bicg = nullptr;       // BiCGStab scalars: outer [nrhs] + inner [nrhs]
    void *h_bicg = nullptr;       // pinned host mirror
    int *d_mask = nullptr;        // per right-hand side masks [2][nrhs]
    int *h_mask = nullptr;
    bool use_graphs = true;       // replay the inner iteration as a CUDA graph when possible
    bool cond_graphs = true;      // the whole inner solve as one graph with a device-decided while loop
    int *d_loop = nullptr;        // that loop's iteration counter (device)
    // host staging for host-pointer calls
    void *d_io = nullptr;
    size_t d_io_bytes = 0;
    // bench buffers
    void *bench_in = nullptr, *bench_out = nullptr;
    size_t bench_bytes = 0;
};

namespace qcd {

// ---- error handling --------------------------------------------------------
int fail(qcd_ctx *c, int code, const std::string &msg);
int cuda_fail(qcd_ctx *c, cudaError_t e, const char *what);
#define QCD_CUDA(ctx, call)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return qcd::cuda_fail(ctx, e_, #call); \
    } while (0)

// ---- launch bookkeeping ------------------------------------------------------
void prof_begin(qcd_ctx *c, int kclass, cudaEvent_t *a);
int prof_end(qcd_ctx *c, int kclass, cudaEvent_t a);
int check_launch(qcd_ctx *c, const char *what);

// ---- memory ------------------------------------------------------------------
// Runs fn() once per call site and device (kernel attributes, constant tables); thread-safe,
// since several host threads may drive contexts at once.  Returns fn's status; a failed
// fn() is tried again on the next call.
template <typename Fn> int once_per_device(std::atomic<unsigned long long> &done, std::mutex &mu, int device, Fn fn) {
    const unsigned long long bit = 1ull << (device & 63);
    if (done.load(std::memory_order_acquire) & bit) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (done.load(std::memory_order_relaxed) & bit) return 0;
    const int rc = fn();
    if (rc == 0) done.fetch_or(bit, std::memory_order_release);
    return rc;
}
int dev_alloc(qcd_ctx *c, void **p, size_t bytes);
void dev_free(qcd_ctx *c, void *p);

// ---- kernels (launchers return QCD_OK or an error) ----------------------------
// layout conversion (layout.cu)
int spinor64_to_internal(qcd_ctx *c, double2 *dst, const double2 *canon, int nrhs);
int spinor64_from_internal(qcd_ctx *c, double2 *canon, const double2 *src, int nrhs);
int spinor32_to_internal(qcd_ctx *c, float4 *dst, const float2 *canon, int nrhs);
int spinor32_from_internal(qcd_ctx *c, float2 *canon, const float4 *src, int nrhs);
int spinor64_to_32(qcd_ctx *c, float4 *dst, const double2 *src, int nrhs);
int spinor32_to_64(qcd_ctx *c, double2 *dst, const float4 *src, int nrhs);
int links_to_internal(qcd_ctx *c, const double2 *canon);

// clover (clover.cu)
int build_clover(qcd_ctx *c, double kappa, double csw);

// operator D (dslash.cu)
struct BicgScalars;
int dslash64(qcd_ctx *c, double2 *out, const double2 *in, int nrhs);
// D in pair-of-FP32 arithmetic: FP32 input (internal layout), FP64 output (internal layout)
// makes the two-row link copy the inner solver's D reads (before any graph capture of it)
int dslash32_prepare(qcd_ctx *c);
int dslash_x2(qcd_ctx *c, double2 *out, const float4 *in, int nrhs);
int dslash32(qcd_ctx *c, float4 *out, const float4 *in, int nrhs);
int dslash16(qcd_ctx *c, float4 *out, const float4 *in, int nrhs);
int dslash12(qcd_ctx *c, float4 *out, const float4 *in, int nrhs);
// FP32 D (two right-hand sides per thread when there are several) fused with the inner
// products of the BiCGStab step that follows: mode 1: red[rhs] = <other, out>, |out|^2; mode 2:
// <out, other>, |out|^2; mode 0: none.  Right-hand sides inactive in gate (may be null) are
// skipped.  Every right-hand side's result is independent of the batch, bit for bit.
int dslash32_dot(qcd_ctx *c, float4 *out, const float4 *in, int nrhs, const float4 *other, int mode, double *red,
                 const BicgScalars *gate);

// SSOR form for a call whose params carry sap_ctas (0: the context's qcd_set_sap_ctas setting);
// rebuilds the SAP plan when it changes (api.cu)
void use_sap_ctas(qcd_ctx *c, int sap_ctas);

// SAP (sap.cu)
// block decomposition valid for the lattice (L % block == 0, L / block even and >= 2,
// block % subblock == 0)
bool sap_geometry_ok(const qcd_ctx *c, const int b[4], const int s[4]);
// host part of a plan (tables in h_*; device pointers left null); QCD_ERR_ARG on bad geometry
int sap_plan_host(const qcd_ctx *c, const int b[4], const int s[4], SapPlan &plan, int min_ctas = 1,
                  bool half = false);
// builds and uploads the plan of this geometry into c->plan (allocates its tables)
int sap_prepare(qcd_ctx *c, const int b[4], const int s[4], bool half);
// drops the cached plan (it is rebuilt on next use)
void sap_invalidate(qcd_ctx *c);
// x = M_SAP v (FP32 internal layout, nrhs right-hand sides); right-hand sides inactive in gate
// (may be null) are skipped.  block_solver 0: ll-SSOR block inverses (nsweep sweeps), work = 2 nrhs
// spinors; 1: even-odd minimal-residual block inverses (nsweep steps), work = 5 nrhs spinors
struct BicgScalars;
int sap_apply(qcd_ctx *c, float4 *x, const float4 *v, float4 *work, double omega, int nsweep, int nsap,
              int nrhs = 1, const BicgScalars *gate = nullptr, int block_solver = 0);
// the even-odd variant with an explicit plan (its block origins)
int sap_apply_eo(qcd_ctx *c, const SapPlan &plan, float4 *x, const float4 *v, float4 *work, int nmr, int nsap,
                 int nrhs, const BicgScalars *gate);
// spinor fields of nrhs right-hand sides the work area of sap_apply needs
inline int sap_work_fields(int block_solver) { return block_solver == 1 ? 5 : 2; }
// the same with an explicit plan whose device tables and records are already in place
int sap_apply_plan(qcd_ctx *c, const SapPlan &plan, float4 *x, const float4 *v, float4 *work, double omega,
                   int nsweep, int nsap, int nrhs = 1, const BicgScalars *gate = nullptr);
// bytes of the device tables of a plan, and their upload into one region (no allocation)
size_t sap_table_bytes(const SapPlan &plan);
int sap_upload_tables(qcd_ctx *c, SapPlan &plan, void *region);
// bytes of one per-site SSOR record (links, clover rows, neighbour codes), of all records of a
// plan, and building them into rec (plan.d_rec is set to rec)
constexpr size_t kSapRecordBytesPerSite = 1200;
size_t sap_record_bytes(const SapPlan &plan);
int sap_build_records(qcd_ctx *c, SapPlan &plan, float *rec);

// RHS-tiled thread form of the SAP cycle (ssor_tile.cu): one CTA per (block, tile of up to
// kTileMaxRhs right-hand sides), one thread per site update, the block spinors of the tile in
// shared memory; per-site records of kTileRecordBytes (FP32) / kTileRecordBytesHalf (FP16)
constexpr int kTileMaxThreads = 256;
constexpr int kTileMinBlocks = 2;  // resident CTAs per SM the register allocation is made for (128 registers)
constexpr int kTileMaxRhs = 8;
constexpr size_t kTileSmemLimit = 200 * 1024;
constexpr size_t kTileSmemPerSm = 228 * 1024;
constexpr int kTileRecordBytes = 672;
constexpr int kTileRecordBytesHalf = 336;
// zero slots of the tile form (one per bank class that an out-of-block hop may need)
constexpr int kTileZeroSlotsHalf = 4;
constexpr int kTileZeroSlots = 2;
// shared memory of a tile CTA with R right-hand sides
size_t tile_smem_bytes(const SapPlan &p, int R);
// tile form: h_tile_pos from the level schedule, the positions of a level ordered against
// shared-memory bank conflicts (needs h_step_site, h_step_ptr, h_site_off, b, vol, half)
void tile_make_positions(SapPlan &p);
// the host check of h_tile_pos that the tile kernel relies on for in-bounds shared memory
bool tile_positions_valid(const SapPlan &p);
int tile_build_records(qcd_ctx *c, const SapPlan &p, void *rec);
int tile_set_attributes(qcd_ctx *c);
// right-hand sides per CTA, threads per CTA and shared memory of a tile launch for nrhs right-hand sides
int tile_choose(const SapPlan &p, int nrhs, int *R, int *threads, size_t *smem);
// x = M_SAP v with the tile form: one launch per colour and cycle, each applying the pending
// hops between blocks, the SSOR sweeps and the residual and solution updates itself; r and y
// are work fields of nrhs right-hand sides
int tile_sap_apply(qcd_ctx *c, const SapPlan &p, float4 *x, const float4 *v, float4 *r, float4 *y, double omega,
                   int nsweep, int nsap, int nrhs, const BicgScalars *gate);

// BLAS (blas.cu), batched: vectors [nrhs][n] complex (double2 or float2), scalars per
// right-hand side in device memory.  A right-hand side whose scalars say inactive is skipped.
struct BicgScalars {
    double2 rho, rho0, alpha, omega, beta;
    double rn2, rhn2, q2;  // |r|^2, |rhat|^2, |rhs|^2
    int active, done, breakdown, iters;
};
enum { SC_INIT = 0, SC_BETA = 1, SC_ALPHA = 2, SC_OMEGA = 3, SC_RHO = 4 };
enum { RED_DOT = 0, RED_DOT_NORM = 1, RED_NORM = 2, RED_DOT_NORMA = 3 };
constexpr int kRedMaxBlocks = 1216;  // 8 x 152 SMs
// out[rhs][3] = Re, Im <a,b> and |b|^2 (DOT_NORM), |a|^2 (NORM, DOT_NORMA); gate: skip inactive rhs
int reduce64(qcd_ctx *c, int kind, const double2 *a, const double2 *b, long n, int nrhs, double *out,
             const BicgScalars *gate);
int reduce32(qcd_ctx *c, int kind, const float2 *a, const float2 *b, long n, int nrhs, double *out,
             const BicgScalars *gate);
// out[rhs][3] = the sums over nblk of the partials [rhs][3][nblk] in c->d_red, in index order
int reduce_partials(qcd_ctx *c, int nblk, int nrhs, double *out);
// the same for ntiles partials [rhs][3][ntiles] anywhere in device memory (two fixed levels:
// contiguous chunks into c->d_red, then those in index order)
int reduce_tiles(qcd_ctx *c, const double *part, long ntiles, int nrhs, double *out);
// one scalar step of BiCGStab (SC_*) for every right-hand side; SC_INIT: gate (may be null)
// deactivates right-hand sides that are inactive in the outer solver
int scalars(qcd_ctx *c, int stage, BicgScalars *S, const double *red, int nrhs, double tol, const BicgScalars *gate);
int blas_zero(qcd_ctx *c, void *p, size_t bytes);
int blas_copy(qcd_ctx *c, void *dst, const void *src, size_t bytes);
// p = r + beta (p - om v)
int blas_p_update64(qcd_ctx *c, double2 *p, const double2 *r, const double2 *v, const BicgScalars *S, long n, int nrhs);
int blas_p_update32(qcd_ctx *c, float2 *p, const float2 *r, const float2 *v, const BicgScalars *S, long n, int nrhs);
// s = r - alpha v
int blas_s_update64(qcd_ctx *c, double2 *s, const double2 *r, const double2 *v, const BicgScalars *S, long n, int nrhs);
int blas_s_update32(qcd_ctx *c, float2 *s, const float2 *r, const float2 *v, const BicgScalars *S, long n, int nrhs);
// x += alpha ph + om sh;  r = s - om t
int blas_xr_update64(qcd_ctx *c, double2 *x, double2 *r, const double2 *ph, const double2 *sh, const double2 *s,
                     const double2 *t, const BicgScalars *S, long n, int nrhs);
int blas_xr_update32(qcd_ctx *c, float2 *x, float2 *r, const float2 *ph, const float2 *sh, const float2 *s,
                     const float2 *t, const BicgScalars *S, long n, int nrhs);
// the same, and out[rhs] = <rh, r>, |r|^2 of the new r (the reduction fused into the update)
int blas_xr_update_dot32(qcd_ctx *c, float2 *x, float2 *r, const float2 *ph, const float2 *sh, const float2 *s,
                         const float2 *t, const float2 *rh, const BicgScalars *S, long n, int nrhs, double *out);
// r = b - w where mask[rhs] (all when mask is null)
int blas_sub64(qcd_ctx *c, double2 *r, const double2 *b, const double2 *w, const int *mask, long n, int nrhs);
// rh = r, p = v = 0 where mask[rhs]
int blas_restart64(qcd_ctx *c, double2 *rh, double2 *p, double2 *v, const double2 *r, const int *mask, long n,
                   int nrhs);

// learned correction (learned.cu)
long learned_weight_count();
int learned_set_weights(qcd_ctx *c, const float2 *w, bool on_device);
int learned_get_weights(qcd_ctx *c, float2 *w_host);
int learned_sync_B(qcd_ctx *c);
// y = N(x), one right-hand side, plane layout FP32
int learned_forward(qcd_ctx *c, float4 *y, const float4 *x, const BicgScalars *gate = nullptr);
// loss of one pair (rho plane layout, eps site layout FP32); gradient added to net.grad
int learned_loss_grad(qcd_ctx *c, const float4 *rho, const float2 *eps, double *loss, float4 *ybuf);
int learned_zero_grad(qcd_ctx *c);
int learned_adam(qcd_ctx *c, float lr);
// out += N(v - D out) per right-hand side; w1, w2 scratch of nrhs fields
// out += N(v - D out) for every right-hand side active in gate (may be null: all)
int learned_correct(qcd_ctx *c, float4 *out, const float4 *v, float4 *w1, float4 *w2, int nrhs,
                    const BicgScalars *gate = nullptr);
// the hidden 8 -> 8 layer on the tcgen05 tensor cores (BF16 site records in and out, or FP32 with
// fp32_io); Bt: its [9][64][64] BF16 B matrices
int learned_layer_tc(qcd_ctx *c, void *y, const void *x, const __nv_bfloat16 *Bt, bool fp32_io,
                     const BicgScalars *gate = nullptr);
// QCD_ERR_TIMEOUT (and the flag cleared) if a tensor-core layer gave up a wait since the last
// check; synchronises the stream
int learned_tc_status(qcd_ctx *c);
int sub_plane(qcd_ctx *c, float4 *r, const float4 *a, const float4 *b, int nrhs);
int plane_to_site(qcd_ctx *c, float2 *out, const float4 *in);

// solver (solver.cu)
// x, b: internal FP64 layout, nrhs right-hand sides
int solve(qcd_ctx *c, double2 *x, const double2 *b, const qcd_params *p, int nrhs, qcd_stats *st);

}  // namespace qcd
