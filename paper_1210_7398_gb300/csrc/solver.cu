// S1: the nested BiCGStab of Sec. 2, batched over right-hand sides.  The outer
// solver is a flexible FP64 BiCGStab on D x = b whose preconditioner is an
// FP32 BiCGStab on D y = q, itself right-preconditioned by M_SAP (Eq. (4)).
// All right-hand sides advance together; each has its own scalars in device
// memory and leaves the iteration (its kernels become no-ops) when it has
// converged or broken down.  The true residual b - D x is recomputed in FP64
// when the recursive one reaches the tolerance; a mismatch, or a breakdown,
// restarts that right-hand side from its true residual (at most 5 restarts).
//
// One inner iteration is a fixed sequence of launches that reads its scalars
// from device memory, so on a capturable stream the inner solve is captured once
// per call as a CUDA graph whose while node repeats the iteration until a kernel
// at its end finds no right-hand side active (or max_inner reached): one graph
// launch and one read of the scalars per inner solve.  Where conditional nodes
// are unavailable the iteration alone is captured and replayed, the host reading
// the active flags after each.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qcd_internal.h"

namespace qcd {

namespace {

#define TRY(call)                 \
    do {                          \
        int rc_ = (call);         \
        if (rc_) return rc_;      \
    } while (0)

struct Ws {
    int nrhs;
    long V;
    // FP64 internal vectors [nrhs][12][V]
    double2 *b, *x, *r, *rh, *p, *v, *s, *t, *ph, *sh, *tmp;
    // FP32 internal vectors [nrhs][6][V]
    float4 *q, *y, *ir, *irh, *ip, *iv, *is, *it, *ipt, *ist, *sapw;
    BicgScalars *So, *Si;  // outer, inner scalars (device)
    BicgScalars *hSo, *hSi;  // pinned host mirrors
    int *mask, *hmask;       // [nrhs] per right-hand side flag (device, host)
    double *red;             // reduction results [nrhs][3]
};

float2 *f2(float4 *a) { return reinterpret_cast<float2 *>(a); }

// the launches of one inner iteration (all scalars on the device)
int inner_iteration(qcd_ctx *c, const Ws &w, const qcd_params *p) {
    const long n = 12 * w.V;
    const int R = w.nrhs;
    TRY(scalars(c, SC_BETA, w.Si, w.red, R, p->inner_tol, nullptr));
    TRY(blas_p_update32(c, f2(w.ip), f2(w.ir), f2(w.iv), w.Si, n, R));
    TRY(sap_apply(c, w.ipt, w.ip, w.sapw, p->omega, p->nsweep, p->nsap, R, w.Si, p->block_solver));
    if (p->learned) TRY(learned_correct(c, w.ipt, w.ip, w.iv, reinterpret_cast<float4 *>(c->net.tmp), R, w.Si));
    TRY(dslash32_dot(c, w.iv, w.ipt, R, w.irh, 1, w.red, w.Si));  // v = D p~; <rh, v>, |v|^2
    TRY(scalars(c, SC_ALPHA, w.Si, w.red, R, p->inner_tol, nullptr));
    TRY(blas_s_update32(c, f2(w.is), f2(w.ir), f2(w.iv), w.Si, n, R));
    TRY(sap_apply(c, w.ist, w.is, w.sapw, p->omega, p->nsweep, p->nsap, R, w.Si, p->block_solver));
    if (p->learned) TRY(learned_correct(c, w.ist, w.is, w.it, reinterpret_cast<float4 *>(c->net.tmp), R, w.Si));
    TRY(dslash32_dot(c, w.it, w.ist, R, w.is, 2, w.red, w.Si));  // t = D s~; <t, s>, |t|^2
    TRY(scalars(c, SC_OMEGA, w.Si, w.red, R, p->inner_tol, nullptr));
    // y += alpha p~ + omega s~, r = s - omega t; <rh, r>, |r|^2
    TRY(blas_xr_update_dot32(c, f2(w.y), f2(w.ir), f2(w.ipt), f2(w.ist), f2(w.is), f2(w.it), f2(w.irh), w.Si, n, R,
                             w.red));
    TRY(scalars(c, SC_RHO, w.Si, w.red, R, p->inner_tol, nullptr));
    return QCD_OK;
}

int any_active(qcd_ctx *c, const Ws &w, BicgScalars *dS, BicgScalars *hS, bool *any, int *iters_total) {
    QCD_CUDA(c, cudaMemcpyAsync(hS, dS, sizeof(BicgScalars) * w.nrhs, cudaMemcpyDeviceToHost, c->stream));
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    *any = false;
    if (iters_total) *iters_total = 0;
    for (int k = 0; k < w.nrhs; k++) {
        *any |= hS[k].active != 0;
        if (iters_total) *iters_total += hS[k].iters;
    }
    return QCD_OK;
}

bool capturable(qcd_ctx *c) {
    if (!c->use_graphs || c->prof.on || c->stream == nullptr) return false;
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st == cudaStreamCaptureStatusNone;
}

// the condition of the inner loop's graph: another iteration while any right-hand side is
// active and fewer than max_inner have run (the counter starts at 0 with each launch)
__global__ void k_inner_continue(cudaGraphConditionalHandle h, const BicgScalars *__restrict__ S, int nrhs,
                                 int *__restrict__ iter, int max_inner) {
    if (threadIdx.x != 0) return;
    int any = 0;
    for (int k = 0; k < nrhs; k++) any |= S[k].active;
    const int it = ++*iter;
    cudaGraphSetConditional(h, (any && it < max_inner) ? 1u : 0u);
}

// The inner solve as one graph: a while node whose body is one inner iteration followed by
// k_inner_continue, so the loop runs on the device with no host round trip per iteration.
// Returns cudaSuccess, or the error of the first graph call that failed (the caller then
// replays the iteration graph from the host instead).
cudaError_t build_loop_graph(qcd_ctx *c, const Ws &w, const qcd_params *p, cudaGraphExec_t *graph, int *rc) {
    *rc = QCD_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const long l0 = c->total_launches;
            *rc = inner_iteration(c, w, p);
            if (!*rc) {
                k_inner_continue<<<1, 32, 0, c->stream>>>(h, w.Si, w.nrhs, c->d_loop, p->max_inner);
                c->total_launches++;
            }
            c->graph_launches = c->total_launches - l0;
            c->total_launches = l0;
            cudaGraph_t captured = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(c->stream, &captured);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e == cudaSuccess && !*rc) e = cudaGraphInstantiate(graph, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// inner FP32 BiCGStab for every right-hand side active in the outer solver:
// y ~ D^{-1} q with right preconditioner M_SAP; returns the iterations summed over rhs
int inner_solve(qcd_ctx *c, const Ws &w, const qcd_params *p, cudaGraphExec_t *graph, int *iters) {
    const long n = 12 * w.V;
    const int R = w.nrhs;
    const size_t bytes = sizeof(float4) * 6 * w.V * R;
    TRY(blas_zero(c, w.y, bytes));
    TRY(blas_copy(c, w.ir, w.q, bytes));
    TRY(blas_copy(c, w.irh, w.q, bytes));
    TRY(blas_zero(c, w.ip, bytes));
    TRY(blas_zero(c, w.iv, bytes));
    TRY(reduce32(c, RED_DOT_NORM, f2(w.irh), f2(w.ir), n, R, w.red, nullptr));
    TRY(scalars(c, SC_INIT, w.Si, w.red, R, p->inner_tol, w.So));
    *iters = 0;
    bool any = false;
    TRY(any_active(c, w, w.Si, w.hSi, &any, nullptr));
    if (any && graph && c->cond_graphs) {
        // the whole loop in one graph launch; the host reads the scalars once at the end
        if (!*graph) {
            int rc = QCD_OK;
            const cudaError_t e = build_loop_graph(c, w, p, graph, &rc);
            if (rc) return rc;
            if (e != cudaSuccess) {
                cudaGetLastError();  // no conditional nodes here: replay the iteration from the host
                if (*graph) cudaGraphExecDestroy(*graph);
                *graph = nullptr;
                c->cond_graphs = false;
            }
        }
        if (*graph) {
            int ran = 0;
            QCD_CUDA(c, cudaMemsetAsync(c->d_loop, 0, sizeof(int), c->stream));
            QCD_CUDA(c, cudaGraphLaunch(*graph, c->stream));
            QCD_CUDA(c, cudaMemcpyAsync(&ran, c->d_loop, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            TRY(any_active(c, w, w.Si, w.hSi, &any, iters));
            c->total_launches += c->graph_launches * ran;
            return QCD_OK;
        }
    }
    for (int it = 0; any && it < p->max_inner; it++) {
        if (graph) {
            if (!*graph) {
                // capture once; the captured launches run only when the graph is launched
                cudaGraph_t g = nullptr;
                const long l0 = c->total_launches;
                QCD_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                int rc = inner_iteration(c, w, p);
                cudaError_t e = cudaStreamEndCapture(c->stream, &g);
                c->graph_launches = c->total_launches - l0;
                c->total_launches = l0;
                if (rc) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
            }
            QCD_CUDA(c, cudaGraphLaunch(*graph, c->stream));
            c->total_launches += c->graph_launches;
        } else {
            TRY(inner_iteration(c, w, p));
        }
        TRY(any_active(c, w, w.Si, w.hSi, &any, iters));
    }
    if (any) TRY(any_active(c, w, w.Si, w.hSi, &any, iters));
    return QCD_OK;
}

int precondition(qcd_ctx *c, const Ws &w, const qcd_params *p, const double2 *in, double2 *out,
                 cudaGraphExec_t *graph, int *iters) {
    TRY(spinor64_to_32(c, w.q, in, w.nrhs));
    TRY(inner_solve(c, w, p, graph, iters));
    TRY(spinor32_to_64(c, out, w.y, w.nrhs));
    return QCD_OK;
}

// out = D y for the outer iteration, y the preconditioner's output (its FP32 original still in
// w.y): the FP64 D; with outer_precision QCD_F32X2 the pair-of-FP32 D of the FP32 original (about
// FP64 accuracy, on the FP32 pipe); with QCD_F32 the FP32 D widened to FP64
int outer_D(qcd_ctx *c, const Ws &w, const qcd_params *p, double2 *out, const double2 *y) {
    if (p->outer_precision == QCD_F32X2) return dslash_x2(c, out, w.y, w.nrhs);
    if (p->outer_precision == QCD_F32) {
        TRY(dslash32(c, w.iv, w.y, w.nrhs));
        return spinor32_to_64(c, out, w.iv, w.nrhs);
    }
    return dslash64(c, out, y, w.nrhs);
}

int ensure(qcd_ctx *c, void **ptr, size_t *have, size_t need) {
    if (*have >= need) return QCD_OK;
    dev_free(c, *ptr);
    *ptr = nullptr;
    *have = 0;
    TRY(dev_alloc(c, ptr, need));
    *have = need;
    return QCD_OK;
}

int workspace(qcd_ctx *c, int nrhs, int block_solver, Ws *w) {
    const long V = c->lat.V;
    const size_t b64 = sizeof(double2) * 12 * V * nrhs, b32 = sizeof(float4) * 6 * V * nrhs;
    TRY(ensure(c, &c->ws64, &c->ws64_bytes, 11 * b64));
    TRY(ensure(c, &c->ws32, &c->ws32_bytes, (10 + sap_work_fields(block_solver)) * b32));
    if (c->red_rhs < nrhs) {
        dev_free(c, c->d_red);
        dev_free(c, c->d_scalars);
        dev_free(c, c->d_bicg);
        dev_free(c, c->d_mask);
        if (c->h_bicg) cudaFreeHost(c->h_bicg);
        if (c->h_mask) cudaFreeHost(c->h_mask);
        c->d_red = c->d_scalars = nullptr;
        c->d_bicg = c->h_bicg = nullptr;
        c->d_mask = c->h_mask = nullptr;
        c->red_rhs = 0;
        dev_free(c, c->d_red_tiles);
        c->d_red_tiles = nullptr;
        TRY(dev_alloc(c, (void **)&c->d_red, sizeof(double) * 3 * kRedMaxBlocks * nrhs));
        TRY(dev_alloc(c, (void **)&c->d_red_tiles, sizeof(double) * 3 * ((V + 127) / 128) * nrhs));
        TRY(dev_alloc(c, (void **)&c->d_scalars, sizeof(double) * 3 * nrhs));
        TRY(dev_alloc(c, &c->d_bicg, sizeof(BicgScalars) * 2 * nrhs));
        TRY(dev_alloc(c, (void **)&c->d_mask, sizeof(int) * nrhs));
        if (cudaMallocHost(&c->h_bicg, sizeof(BicgScalars) * 2 * nrhs) != cudaSuccess ||
            cudaMallocHost((void **)&c->h_mask, sizeof(int) * nrhs) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, QCD_ERR_OOM, "cudaMallocHost failed");
        }
        c->red_rhs = nrhs;
    }
    if (!c->d_loop) TRY(dev_alloc(c, (void **)&c->d_loop, sizeof(int)));
    w->nrhs = nrhs;
    w->V = V;
    double2 *base = (double2 *)c->ws64;
    double2 **v64[] = {&w->b, &w->x, &w->r, &w->rh, &w->p, &w->v, &w->s, &w->t, &w->ph, &w->sh, &w->tmp};
    for (int k = 0; k < 11; k++) *v64[k] = base + (size_t)k * 12 * V * nrhs;
    float4 *b32p = (float4 *)c->ws32;
    float4 **v32[] = {&w->q, &w->y, &w->ir, &w->irh, &w->ip, &w->iv, &w->is, &w->it, &w->ipt, &w->ist, &w->sapw};
    for (int k = 0; k < 11; k++) *v32[k] = b32p + (size_t)k * 6 * V * nrhs;  // sapw spans the SAP work fields
    w->So = (BicgScalars *)c->d_bicg;
    w->Si = w->So + nrhs;
    w->hSo = (BicgScalars *)c->h_bicg;
    w->hSi = w->hSo + nrhs;
    w->mask = c->d_mask;
    w->hmask = c->h_mask;
    w->red = c->d_scalars;
    return QCD_OK;
}

}  // namespace

int solve(qcd_ctx *c, double2 *x, const double2 *b, const qcd_params *p, int nrhs, qcd_stats *st) {
    Ws w;
    TRY(workspace(c, nrhs, p->block_solver, &w));
    TRY(dslash32_prepare(c));  // the inner D's link copy, made here rather than inside a graph capture
    const long n = 12 * w.V;
    const size_t b64 = sizeof(double2) * n * nrhs;
    const int R = nrhs;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t *gp = capturable(c) ? &graph : nullptr;
    struct GraphGuard {
        cudaGraphExec_t *g;
        ~GraphGuard() {
            if (g && *g) cudaGraphExecDestroy(*g);
        }
    } guard{gp};

    TRY(blas_copy(c, w.b, b, b64));
    TRY(blas_copy(c, w.x, x, b64));
    // |b|^2 and |x0|^2 per rhs
    TRY(reduce64(c, RED_NORM, w.b, nullptr, n, R, w.red, nullptr));
    std::vector<double> bn2(R), h(6 * R);
    QCD_CUDA(c, cudaMemcpyAsync(h.data(), w.red, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, c->stream));
    TRY(reduce64(c, RED_NORM, w.x, nullptr, n, R, w.red, nullptr));
    QCD_CUDA(c, cudaMemcpyAsync(h.data() + 3 * R, w.red, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, c->stream));
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    bool x0_zero = true;
    for (int k = 0; k < R; k++) {
        bn2[k] = h[3 * k + 2];
        x0_zero = x0_zero && h[3 * (R + k) + 2] == 0.0;
    }
    // r = b - D x (r = b when every initial guess is zero); rh = r; p = v = 0
    if (x0_zero) {
        TRY(blas_copy(c, w.r, w.b, b64));
    } else {
        TRY(dslash64(c, w.tmp, w.x, R));
        TRY(blas_sub64(c, w.r, w.b, w.tmp, nullptr, n, R));
    }
    TRY(blas_copy(c, w.rh, w.r, b64));
    TRY(blas_zero(c, w.p, b64));
    TRY(blas_zero(c, w.v, b64));
    TRY(reduce64(c, RED_DOT_NORM, w.rh, w.r, n, R, w.red, nullptr));
    TRY(scalars(c, SC_INIT, w.So, w.red, R, p->tol, nullptr));
    {
        // the outer tolerance is relative to |b|, not to the initial residual
        QCD_CUDA(c, cudaMemcpyAsync(w.hSo, w.So, sizeof(BicgScalars) * R, cudaMemcpyDeviceToHost, c->stream));
        QCD_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int k = 0; k < R; k++) w.hSo[k].q2 = bn2[k];
        QCD_CUDA(c, cudaMemcpyAsync(w.So, w.hSo, sizeof(BicgScalars) * R, cudaMemcpyHostToDevice, c->stream));
    }
    // per rhs bookkeeping on the host
    std::vector<int> restarts(R, 0), status(R, QCD_ERR_NOCONV);
    std::vector<double> relres(R, 0.0);
    int outer = 0, inner = 0;
    auto true_residual = [&](const int *hmask, int *any_masked) -> int {
        // r_true = b - D x for the masked rhs, and its norm
        int m = 0;
        for (int k = 0; k < R; k++) m |= hmask[k];
        *any_masked = m;
        if (!m) return QCD_OK;
        QCD_CUDA(c, cudaMemcpyAsync(w.mask, hmask, sizeof(int) * R, cudaMemcpyHostToDevice, c->stream));
        TRY(dslash64(c, w.tmp, w.x, R));
        TRY(blas_sub64(c, w.r, w.b, w.tmp, w.mask, n, R));
        TRY(reduce64(c, RED_NORM, w.r, nullptr, n, R, w.red, nullptr));
        std::vector<double> h(3 * R);
        QCD_CUDA(c, cudaMemcpyAsync(h.data(), w.red, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, c->stream));
        QCD_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int k = 0; k < R; k++)
            if (hmask[k])
                relres[k] = !std::isfinite(bn2[k]) ? INFINITY : bn2[k] > 0 ? std::sqrt(h[3 * k + 2] / bn2[k]) : 0.0;
        return QCD_OK;
    };
    // rhs with b = 0 are solved by x = 0; rhs whose initial residual is small enough are done;
    // rhs holding a non-finite value are settled (not converged) at once
    {
        bool any = false;
        TRY(any_active(c, w, w.So, w.hSo, &any, nullptr));
        for (int k = 0; k < R; k++) {
            w.hmask[k] = 0;
            if (bn2[k] == 0) {
                status[k] = QCD_OK;
            } else if (!std::isfinite(bn2[k]) || !w.hSo[k].active || w.hSo[k].rn2 <= p->tol * p->tol * bn2[k]) {
                w.hmask[k] = 1;
            }
        }
    }
    std::vector<int> h_active(R, 0);
    for (int k = 0; k < R; k++) h_active[k] = w.hSo[k].active && bn2[k] > 0;
    while (true) {
        // settle the rhs flagged in hmask: check the true residual, finish or restart them
        int any_masked = 0;
        TRY(true_residual(w.hmask, &any_masked));
        if (any_masked) {
            std::vector<int> restart(R, 0);
            for (int k = 0; k < R; k++) {
                if (!w.hmask[k]) continue;
                if (!std::isfinite(bn2[k])) {  // never iterated, never reported converged
                    status[k] = QCD_ERR_NOCONV;
                    h_active[k] = 0;
                } else if (relres[k] <= p->tol) {
                    status[k] = QCD_OK;
                    h_active[k] = 0;
                } else if (++restarts[k] > 5 || outer >= p->max_outer) {
                    status[k] = (restarts[k] > 5 && w.hSo[k].breakdown) ? QCD_ERR_BREAKDOWN : QCD_ERR_NOCONV;
                    h_active[k] = 0;
                } else {
                    restart[k] = 1;
                    h_active[k] = 1;
                }
            }
            int any_restart = 0;
            for (int k = 0; k < R; k++) any_restart |= restart[k];
            if (any_restart) {
                QCD_CUDA(c, cudaMemcpyAsync(w.mask, restart.data(), sizeof(int) * R, cudaMemcpyHostToDevice, c->stream));
                TRY(blas_restart64(c, w.rh, w.p, w.v, w.r, w.mask, n, R));
            }
            // re-initialise the scalars of restarted rhs, keep the others' state; deactivate the finished ones
            TRY(reduce64(c, RED_DOT_NORM, w.rh, w.r, n, R, w.red, nullptr));
            QCD_CUDA(c, cudaMemcpyAsync(w.hSo, w.So, sizeof(BicgScalars) * R, cudaMemcpyDeviceToHost, c->stream));
            QCD_CUDA(c, cudaStreamSynchronize(c->stream));
            std::vector<double> h(3 * R);
            QCD_CUDA(c, cudaMemcpyAsync(h.data(), w.red, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, c->stream));
            QCD_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int k = 0; k < R; k++) {
                BicgScalars &s = w.hSo[k];
                if (restart[k]) {
                    s.rho = make_double2(h[3 * k], h[3 * k + 1]);
                    s.rn2 = s.rhn2 = h[3 * k + 2];
                    s.q2 = bn2[k];
                    s.rho0 = s.alpha = s.omega = make_double2(1.0, 0.0);
                    s.breakdown = s.done = 0;
                }
                s.active = h_active[k];
            }
            QCD_CUDA(c, cudaMemcpyAsync(w.So, w.hSo, sizeof(BicgScalars) * R, cudaMemcpyHostToDevice, c->stream));
        }
        bool any = false;
        for (int k = 0; k < R; k++) any |= h_active[k] != 0;
        if (!any || outer >= p->max_outer) break;
        // one outer iteration for every active rhs
        if (c->inject_breakdown > 0) {
            // test hook: rho = 0 in the scalar state of every active rhs, as a vanishing <rh, r>
            // would leave it; the beta step then reports the breakdown
            c->inject_breakdown--;
            QCD_CUDA(c, cudaMemcpyAsync(w.hSo, w.So, sizeof(BicgScalars) * R, cudaMemcpyDeviceToHost, c->stream));
            QCD_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int k = 0; k < R; k++)
                if (w.hSo[k].active) w.hSo[k].rho = make_double2(0.0, 0.0);
            QCD_CUDA(c, cudaMemcpyAsync(w.So, w.hSo, sizeof(BicgScalars) * R, cudaMemcpyHostToDevice, c->stream));
        }
        TRY(scalars(c, SC_BETA, w.So, w.red, R, p->tol, nullptr));
        TRY(blas_p_update64(c, w.p, w.r, w.v, w.So, n, R));
        int its = 0;
        TRY(precondition(c, w, p, w.p, w.ph, gp, &its));
        inner += its;
        TRY(outer_D(c, w, p, w.v, w.ph));
        TRY(reduce64(c, RED_DOT_NORM, w.rh, w.v, n, R, w.red, w.So));
        TRY(scalars(c, SC_ALPHA, w.So, w.red, R, p->tol, nullptr));
        TRY(blas_s_update64(c, w.s, w.r, w.v, w.So, n, R));
        TRY(precondition(c, w, p, w.s, w.sh, gp, &its));
        inner += its;
        TRY(outer_D(c, w, p, w.t, w.sh));
        TRY(reduce64(c, RED_DOT_NORMA, w.t, w.s, n, R, w.red, w.So));
        TRY(scalars(c, SC_OMEGA, w.So, w.red, R, p->tol, nullptr));
        TRY(blas_xr_update64(c, w.x, w.r, w.ph, w.sh, w.s, w.t, w.So, n, R));
        TRY(reduce64(c, RED_DOT_NORM, w.rh, w.r, n, R, w.red, w.So));
        TRY(scalars(c, SC_RHO, w.So, w.red, R, p->tol, nullptr));
        outer++;
        // rhs that left the outer iteration (converged recursively or broke down) get their true residual checked
        bool dummy = false;
        TRY(any_active(c, w, w.So, w.hSo, &dummy, nullptr));
        for (int k = 0; k < R; k++) {
            w.hmask[k] = (h_active[k] && !w.hSo[k].active) ? 1 : 0;
            if (h_active[k] && w.hSo[k].active && outer >= p->max_outer) w.hmask[k] = 1;
        }
    }
    // rhs still unsettled (max_outer): their true residual
    {
        int any_masked = 0;
        for (int k = 0; k < R; k++) w.hmask[k] = status[k] != QCD_OK ? 1 : 0;
        TRY(true_residual(w.hmask, &any_masked));
    }
    TRY(blas_copy(c, x, w.x, b64));
    int worst = QCD_OK;
    for (int k = 0; k < R; k++)
        if (status[k] != QCD_OK) worst = (worst == QCD_OK || status[k] == QCD_ERR_BREAKDOWN) ? status[k] : worst;
    if (st) {
        st->outer_iters += outer;
        st->inner_iters += inner;
        int rs = 0;
        for (int k = 0; k < R; k++) rs += restarts[k];
        st->restarts += rs;
        for (int k = 0; k < R; k++) st->true_rel_res = std::max(st->true_rel_res, relres[k]);
        if (st->status == QCD_OK) st->status = worst;
    }
    return worst;
}

}  // namespace qcd
