// C ABI of the solver library (declared in include/qcd.h): argument checks,
// context and memory management, host/device staging and the launch
// bookkeeping used for measurement.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "qcd_internal.h"

namespace qcd {

int fail(qcd_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(qcd_ctx *c, cudaError_t e, const char *what) {
    if (c) {
        c->err = std::string(what) + ": " + cudaGetErrorString(e);
        c->poisoned = true;
    }
    if (e == cudaErrorMemoryAllocation) return QCD_ERR_OOM;
    return QCD_ERR_CUDA;
}

static cudaEvent_t ev_get(qcd_ctx *c) {
    if (!c->prof.pool.empty()) {
        cudaEvent_t e = c->prof.pool.back();
        c->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(qcd_ctx *c, int kclass, cudaEvent_t *a) {
    (void)kclass;
    *a = nullptr;
    if (c->prof.on) {
        *a = ev_get(c);
        cudaEventRecord(*a, c->stream);
    }
}

int check_launch(qcd_ctx *c, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return QCD_OK;
}

int prof_end(qcd_ctx *c, int kclass, cudaEvent_t a) {
    c->total_launches++;
    c->prof.launches[kclass]++;
    int rc = check_launch(c, "kernel launch");
    if (rc) return rc;
    if (c->prof.on && a) {
        cudaEvent_t b = ev_get(c);
        cudaEventRecord(b, c->stream);
        c->prof.pending.push_back({kclass, a, b});
    }
    return QCD_OK;
}

static int prof_collect(qcd_ctx *c) {
    if (c->prof.pending.empty()) return QCD_OK;
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto &p : c->prof.pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        c->prof.ms[p.kclass] += ms;
        c->prof.pool.push_back(p.a);
        c->prof.pool.push_back(p.b);
    }
    c->prof.pending.clear();
    return QCD_OK;
}

int dev_alloc(qcd_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, QCD_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    return QCD_OK;
}

void dev_free(qcd_ctx *c, void *p) {
    (void)c;
    if (p) cudaFree(p);
}

}  // namespace qcd

using namespace qcd;

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ready(qcd_ctx *c) {
    if (!c) return QCD_ERR_ARG;
    if (c->poisoned) return fail(c, QCD_ERR_STATE, "context poisoned by an earlier CUDA error: " + c->err);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return QCD_OK;
}

int need_clover(qcd_ctx *c) {
    if (!c->have_clover) return fail(c, QCD_ERR_STATE, "qcd_build_clover must be called first");
    return QCD_OK;
}

int ensure_io(qcd_ctx *c, size_t bytes) {
    if (c->d_io_bytes >= bytes) return QCD_OK;
    dev_free(c, c->d_io);
    c->d_io = nullptr;
    c->d_io_bytes = 0;
    int rc = dev_alloc(c, &c->d_io, bytes);
    if (rc) return rc;
    c->d_io_bytes = bytes;
    return QCD_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

void qcd::use_sap_ctas(qcd_ctx *c, int sap_ctas) {
    const int eff = sap_ctas != 0 ? sap_ctas : c->sap_ctas_user;
    if (eff != c->sap_min_ctas) {
        sap_invalidate(c);
        c->sap_min_ctas = eff;
    }
}

namespace {

int check_params(qcd_ctx *c, const qcd_params *p) {
    if (!p) return fail(c, QCD_ERR_ARG, "params is NULL");
    if (!(p->omega > 0 && p->omega < 2)) return fail(c, QCD_ERR_ARG, "omega must lie in (0, 2)");
    if (p->nsweep < 1 || p->nsap < 1) return fail(c, QCD_ERR_ARG, "nsweep and nsap must be >= 1");
    if (p->sap_storage != QCD_F32 && p->sap_storage != QCD_F16)
        return fail(c, QCD_ERR_ARG, "sap_storage must be QCD_F32 or QCD_F16");
    if (p->learned < 0 || p->learned > 2) return fail(c, QCD_ERR_ARG, "learned must be 0, 1 or 2");
    if (p->learned && !c->net.ready) return fail(c, QCD_ERR_STATE, "learned != 0 needs qcd_learned_set_weights");
    if (p->bc_t != c->bc_t) return fail(c, QCD_ERR_ARG, "params.bc_t differs from the context boundary condition");
    if (p->kappa != c->kappa || p->csw != c->csw)
        return fail(c, QCD_ERR_ARG, "params.kappa/csw differ from the clover field built");
    if (p->sap_ctas < -2 || p->sap_ctas > 16) return fail(c, QCD_ERR_ARG, "sap_ctas must lie in -2..16");
    if (p->block_solver < 0 || p->block_solver > 1) return fail(c, QCD_ERR_ARG, "block_solver must be 0 or 1");
    if (p->outer_precision != QCD_F64 && p->outer_precision != QCD_F32 && p->outer_precision != QCD_F32X2)
        return fail(c, QCD_ERR_ARG, "outer_precision must be QCD_F64, QCD_F32 or QCD_F32X2");
    if (p->block_solver == 1 && (p->sap_storage != QCD_F32 || p->learned != 0))
        return fail(c, QCD_ERR_ARG, "block_solver 1 needs sap_storage QCD_F32 and learned 0");
    use_sap_ctas(c, p->sap_ctas);
    return QCD_OK;
}

}  // namespace

extern "C" {

int qcd_create(qcd_ctx **out, const int dims[4], void *stream) {
    if (!out || !dims) return QCD_ERR_ARG;
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; m++) {
        if (dims[m] < 2 || dims[m] > 4096) return QCD_ERR_ARG;
        V *= dims[m];
    }
    if (V > (1L << 31)) return QCD_ERR_ARG;
    qcd_ctx *c = new (std::nothrow) qcd_ctx();
    if (!c) return QCD_ERR_OOM;
    static std::atomic<long> next_uid{1};
    c->uid = next_uid.fetch_add(1);
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)stream;
    for (int m = 0; m < 4; m++) c->lat.L[m] = dims[m];
    c->lat.V = V;
    int rc = QCD_OK;
    if (!rc) rc = dev_alloc(c, (void **)&c->U64, sizeof(double2) * 36 * V);
    if (!rc) rc = dev_alloc(c, (void **)&c->U32, sizeof(float2) * 36 * V);
    if (!rc) rc = dev_alloc(c, (void **)&c->F64, sizeof(double2) * 36 * V);
    if (!rc) rc = dev_alloc(c, (void **)&c->F32, sizeof(float4) * 18 * V);
    if (!rc) rc = dev_alloc(c, (void **)&c->d_status, sizeof(int) * 16);
    if (!rc && cudaMemset(c->d_status, 0, sizeof(int) * 16) != cudaSuccess) {
        cudaGetLastError();
        rc = QCD_ERR_CUDA;
    }
    if (!rc && cudaMallocHost((void **)&c->h_scalars, sizeof(double) * 16) != cudaSuccess) {
        cudaGetLastError();
        rc = QCD_ERR_OOM;
    }
    if (rc) {
        qcd_destroy(c);
        return rc;
    }
    *out = c;
    return QCD_OK;
}

void qcd_destroy(qcd_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    void *bufs[] = {c->net.W, c->net.grad, c->net.m, c->net.v, c->net.B, c->net.P, c->net.scal, c->net.act,
                    c->net.pairs,
                    c->U64, c->U32, c->F64, c->F32, c->U16, c->F16, c->U12, c->Ux2, c->Fx2, c->d_status, c->d_red, c->d_red_tiles, c->d_scalars, c->d_bicg, c->d_mask,
                    c->d_loop, c->ws64, c->ws32,
                    c->d_io, c->bench_in, c->bench_out, c->plan.d_origin[0] /* the plan's table region */,
                    c->plan.d_rec};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (c->h_scalars) cudaFreeHost(c->h_scalars);
    if (c->h_bicg) cudaFreeHost(c->h_bicg);
    if (c->h_mask) cudaFreeHost(c->h_mask);
    for (auto &p : c->prof.pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->prof.pool) cudaEventDestroy(e);
    cudaGetLastError();
    delete c;
}

const char *qcd_last_error(const qcd_ctx *c) {
    if (!c) return "null context";
    return c->err.c_str();
}

int qcd_set_boundary(qcd_ctx *c, int bc_t) {
    int rc = ready(c);
    if (rc) return rc;
    if (bc_t != 1 && bc_t != -1) return fail(c, QCD_ERR_ARG, "bc_t must be +1 or -1");
    c->bc_t = bc_t;
    return QCD_OK;
}

int qcd_load_gauge(qcd_ctx *c, const double *U, int on_device) {
    int rc = ready(c);
    if (rc) return rc;
    if (!U) return fail(c, QCD_ERR_ARG, "U is NULL");
    const size_t bytes = sizeof(double2) * 36 * c->lat.V;
    const double2 *src = (const double2 *)U;
    if (!on_device) {
        if ((rc = ensure_io(c, bytes))) return rc;
        QCD_CUDA(c, cudaMemcpyAsync(c->d_io, U, bytes, cudaMemcpyHostToDevice, c->stream));
        src = (const double2 *)c->d_io;
    } else if (!aligned16(U)) {
        return fail(c, QCD_ERR_ARG, "device U must be 16-byte aligned");
    }
    if ((rc = links_to_internal(c, src))) return rc;
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_gauge = true;
    c->field_version++;
    c->have_clover = false;
    return QCD_OK;
}

int qcd_build_clover(qcd_ctx *c, double kappa, double csw) {
    int rc = ready(c);
    if (rc) return rc;
    if (!c->have_gauge) return fail(c, QCD_ERR_STATE, "qcd_load_gauge must be called first");
    if (!(kappa > 0 && kappa < 1) || !(csw >= 0 && csw < 100)) return fail(c, QCD_ERR_ARG, "kappa or csw out of range");
    c->have_clover = false;
    if ((rc = build_clover(c, kappa, csw))) return rc;
    c->kappa = kappa;
    c->csw = csw;
    c->have_clover = true;
    c->field_version++;
    return QCD_OK;
}

int qcd_apply_D(qcd_ctx *c, void *out, const void *in, int prec, int nrhs) {
    int rc = ready(c);
    if (rc) return rc;
    if ((rc = need_clover(c))) return rc;
    if (!out || !in || nrhs < 1 ||
        (prec != QCD_F64 && prec != QCD_F32 && prec != QCD_F16 && prec != QCD_F32_SU3 && prec != QCD_F32X2))
        return fail(c, QCD_ERR_ARG, "qcd_apply_D: bad pointer, nrhs or precision");
    const long V = c->lat.V;
    const size_t elem = (prec == QCD_F64) ? 16 : 8;
    const size_t bytes = elem * 12 * V * nrhs;
    const size_t obytes = (prec == QCD_F32X2 ? 16 : elem) * 12 * V * nrhs;  // F32X2: complex64 in, complex128 out
    const bool dev_in = is_device_ptr(in), dev_out = is_device_ptr(out);
    if ((dev_in && !aligned16(in)) || (dev_out && !aligned16(out)))
        return fail(c, QCD_ERR_ARG, "device spinors must be 16-byte aligned");
    if ((rc = ensure_io(c, 3 * obytes))) return rc;  // internal in, internal out, staged host in / out
    char *io = (char *)c->d_io;
    const void *din = in;
    void *dout = dev_out ? out : io + 2 * obytes;
    if (!dev_in) {
        QCD_CUDA(c, cudaMemcpyAsync(io + 2 * obytes, in, bytes, cudaMemcpyHostToDevice, c->stream));
        din = io + 2 * obytes;
    }
    if (prec == QCD_F32X2) {
        float4 *a = (float4 *)io;
        double2 *b = (double2 *)(io + obytes);
        if ((rc = spinor32_to_internal(c, a, (const float2 *)din, nrhs))) return rc;
        if ((rc = dslash_x2(c, b, a, nrhs))) return rc;
        if ((rc = spinor64_from_internal(c, (double2 *)dout, b, nrhs))) return rc;
    } else if (prec == QCD_F64) {
        double2 *a = (double2 *)io, *b = (double2 *)(io + bytes);
        if ((rc = spinor64_to_internal(c, a, (const double2 *)din, nrhs))) return rc;
        if ((rc = dslash64(c, b, a, nrhs))) return rc;
        if ((rc = spinor64_from_internal(c, (double2 *)dout, b, nrhs))) return rc;
    } else {
        float4 *a = (float4 *)io, *b = (float4 *)(io + bytes);
        if ((rc = spinor32_to_internal(c, a, (const float2 *)din, nrhs))) return rc;
        if ((rc = (prec == QCD_F16 ? dslash16 : prec == QCD_F32_SU3 ? dslash12 : dslash32)(c, b, a, nrhs))) return rc;
        if ((rc = spinor32_from_internal(c, (float2 *)dout, b, nrhs))) return rc;
    }
    if (!dev_out) QCD_CUDA(c, cudaMemcpyAsync(out, dout, obytes, cudaMemcpyDeviceToHost, c->stream));
    if (!dev_in || !dev_out) QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    return QCD_OK;
}

int qcd_sap_precondition(qcd_ctx *c, float *out, const float *in, const qcd_params *p, int nrhs) {
    int rc = ready(c);
    if (rc) return rc;
    if ((rc = need_clover(c))) return rc;
    if (!out || !in || nrhs < 1) return fail(c, QCD_ERR_ARG, "qcd_sap_precondition: bad pointer or nrhs");
    if ((rc = check_params(c, p))) return rc;
    if ((rc = sap_prepare(c, p->block, p->subblock, p->sap_storage == QCD_F16))) return rc;
    const long V = c->lat.V;
    const size_t bytes = 8 * 12 * V;  // one complex64 right-hand side
    const bool dev_in = is_device_ptr(in), dev_out = is_device_ptr(out);
    if ((dev_in && !aligned16(in)) || (dev_out && !aligned16(out)))
        return fail(c, QCD_ERR_ARG, "device spinors must be 16-byte aligned");
    // io: v, x (internal, nrhs each), work (2 or 5 nrhs), staging (1); all right-hand sides go
    // through one batched SAP application
    const int nw = sap_work_fields(p->block_solver);
    if ((rc = ensure_io(c, ((2 + nw) * (size_t)nrhs + 1) * bytes))) return rc;
    char *io = (char *)c->d_io;
    float4 *v = (float4 *)io, *x = (float4 *)(io + nrhs * bytes), *work = (float4 *)(io + 2 * nrhs * bytes);
    char *stage = io + (2 + nw) * nrhs * bytes;
    if (dev_in) {
        if ((rc = spinor32_to_internal(c, v, (const float2 *)in, nrhs))) return rc;
    } else {
        for (int k = 0; k < nrhs; k++) {
            QCD_CUDA(c, cudaMemcpyAsync(stage, (const char *)in + k * bytes, bytes, cudaMemcpyHostToDevice, c->stream));
            if ((rc = spinor32_to_internal(c, v + k * 6 * V, (const float2 *)stage, 1))) return rc;
        }
    }
    if ((rc = sap_apply(c, x, v, work, p->omega, p->nsweep, p->nsap, nrhs, nullptr, p->block_solver))) return rc;
    if (dev_out) {
        if ((rc = spinor32_from_internal(c, (float2 *)out, x, nrhs))) return rc;
    } else {
        for (int k = 0; k < nrhs; k++) {
            if ((rc = spinor32_from_internal(c, (float2 *)stage, x + k * 6 * V, 1))) return rc;
            QCD_CUDA(c, cudaMemcpyAsync((char *)out + k * bytes, stage, bytes, cudaMemcpyDeviceToHost, c->stream));
            QCD_CUDA(c, cudaStreamSynchronize(c->stream));
        }
    }
    if (!dev_in) QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    return QCD_OK;
}

int qcd_solve(qcd_ctx *c, double *x, const double *b, const qcd_params *p, int nrhs, qcd_stats *st) {
    auto t0 = std::chrono::steady_clock::now();
    int rc = ready(c);
    if (rc) return rc;
    if ((rc = need_clover(c))) return rc;
    if (!x || !b || nrhs < 1) return fail(c, QCD_ERR_ARG, "qcd_solve: bad pointer or nrhs");
    if ((rc = check_params(c, p))) return rc;
    if (!(p->tol > 0) || !(p->inner_tol > 0) || p->max_outer < 1 || p->max_inner < 1)
        return fail(c, QCD_ERR_ARG, "tol, inner_tol, max_outer, max_inner must be positive");
    if (p->rhs_group < 0) return fail(c, QCD_ERR_ARG, "rhs_group must be >= 0");
    if ((rc = sap_prepare(c, p->block, p->subblock, p->sap_storage == QCD_F16))) return rc;
    qcd_stats local;
    std::memset(&local, 0, sizeof(local));
    local.status = QCD_OK;
    const long V = c->lat.V;
    const size_t per = 16 * 12 * (size_t)V;  // one right-hand side, complex128
    const bool dev_x = is_device_ptr(x), dev_b = is_device_ptr(b);
    if ((dev_x && !aligned16(x)) || (dev_b && !aligned16(b)))
        return fail(c, QCD_ERR_ARG, "device spinors must be 16-byte aligned");
    // right-hand sides per group: as asked, or as many as the free device memory holds (the
    // solver's FP64 and FP32 vectors, the internal copies of x and b, host staging)
    int g = p->rhs_group > 0 ? std::min(p->rhs_group, nrhs) : nrhs;
    if (p->rhs_group == 0) {
        size_t fr = 0, tot = 0;
        QCD_CUDA(c, cudaMemGetInfo(&fr, &tot));
        const size_t held = c->ws64_bytes + c->ws32_bytes + c->d_io_bytes;
        const size_t margin = (size_t)1 << 30;
        const size_t avail = fr + held > margin + tot / 50 ? fr + held - margin - tot / 50 : 0;
        const size_t need = 16 * 12 * (size_t)V * 11 + 16 * 6 * (size_t)V * (10 + sap_work_fields(p->block_solver)) +
                            per * (dev_x && dev_b ? 2 : 4);
        g = (int)std::max<size_t>(1, std::min<size_t>((size_t)nrhs, avail / need));
    }
    // learned = 1 falls back to plain SAP when the last evaluation found the correction slower
    qcd_params pe = *p;
    pe.learned = (p->learned == 2 || (p->learned == 1 && c->net.verdict != 0)) ? 1 : 0;
    // device time per kernel class during this call (kernel profiling on)
    double ms0[QCD_K_COUNT] = {};
    if (c->prof.on) {
        if ((rc = prof_collect(c))) return rc;
        std::memcpy(ms0, c->prof.ms, sizeof(ms0));
    }
    int status = QCD_OK;
    for (int k0 = 0; k0 < nrhs; k0 += g) {
        const int n = std::min(g, nrhs - k0);
        const size_t bytes = per * n;
        if ((rc = ensure_io(c, 4 * per * g))) return rc;
        char *io = (char *)c->d_io;
        double2 *xi = (double2 *)io, *bi = (double2 *)(io + bytes);
        char *sx = io + 2 * bytes, *sb = io + 3 * bytes;
        const char *bsrc = (const char *)b + per * k0, *xsrc = (const char *)x + per * k0;
        if (!dev_b) {
            QCD_CUDA(c, cudaMemcpyAsync(sb, bsrc, bytes, cudaMemcpyHostToDevice, c->stream));
            bsrc = sb;
        }
        if (!dev_x) {
            QCD_CUDA(c, cudaMemcpyAsync(sx, xsrc, bytes, cudaMemcpyHostToDevice, c->stream));
            xsrc = sx;
        }
        if ((rc = spinor64_to_internal(c, bi, (const double2 *)bsrc, n))) return rc;
        if ((rc = spinor64_to_internal(c, xi, (const double2 *)xsrc, n))) return rc;
        const int s = solve(c, xi, bi, &pe, n, &local);
        if (s == QCD_ERR_CUDA || s == QCD_ERR_OOM || s == QCD_ERR_STATE || s == QCD_ERR_ARG) return s;
        if (s != QCD_OK && (status == QCD_OK || s == QCD_ERR_BREAKDOWN)) status = s;
        char *xdst = dev_x ? (char *)x + per * k0 : sx;
        if ((rc = spinor64_from_internal(c, (double2 *)xdst, xi, n))) return rc;
        if (!dev_x) QCD_CUDA(c, cudaMemcpyAsync((char *)x + per * k0, sx, bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->prof.on) {
        if ((rc = prof_collect(c))) return rc;
        local.ms_dslash = c->prof.ms[QCD_K_DSLASH32] - ms0[QCD_K_DSLASH32] + c->prof.ms[QCD_K_DSLASH64] - ms0[QCD_K_DSLASH64];
        local.ms_sap = c->prof.ms[QCD_K_SSOR] - ms0[QCD_K_SSOR] + c->prof.ms[QCD_K_SAPHOP] - ms0[QCD_K_SAPHOP];
    }
    if (p->learned && (rc = learned_tc_status(c))) return rc;
    local.status = status;
    local.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st) *st = local;
    if (status != QCD_OK) {
        if (status == QCD_ERR_NOCONV) c->err = "not converged within max_outer (or a right-hand side is not finite)";
        else if (status == QCD_ERR_BREAKDOWN) c->err = "BiCGStab breakdown not cured by restarts";
    }
    return status;
}

int qcd_solve_multi(int n, qcd_ctx *const *ctxs, double *const *x, const double *const *b, const qcd_params *params,
                    const int *nrhs, qcd_stats *stats) {
    if (n < 1 || !ctxs || !x || !b || !params || !nrhs) return QCD_ERR_ARG;
    for (int i = 0; i < n; i++) {
        if (!ctxs[i]) return QCD_ERR_ARG;
        if (!ctxs[i]->stream) return fail(ctxs[i], QCD_ERR_ARG, "qcd_solve_multi: each context needs its own stream");
        for (int j = 0; j < i; j++)
            if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream)
                return fail(ctxs[i], QCD_ERR_ARG, "qcd_solve_multi: contexts and streams must be distinct");
    }
    std::vector<int> rc(n, QCD_OK);
    std::vector<qcd_stats> st(n);
    auto one = [&](int i) {
        cudaSetDevice(ctxs[i]->device);
        std::memset(&st[i], 0, sizeof(qcd_stats));
        rc[i] = qcd_solve(ctxs[i], x[i], b[i], &params[i], nrhs[i], &st[i]);
    };
    std::vector<std::thread> th;
    th.reserve(n - 1);
    for (int i = 1; i < n; i++) th.emplace_back(one, i);
    one(0);
    for (auto &t : th) t.join();
    if (stats)
        for (int i = 0; i < n; i++) stats[i] = st[i];
    for (int i = 0; i < n; i++)
        if (rc[i] != QCD_OK) return rc[i];
    return QCD_OK;
}

int qcd_set_graphs(qcd_ctx *c, int on) {
    int rc = ready(c);
    if (rc) return rc;
    c->use_graphs = on != 0;
    return QCD_OK;
}

int qcd_set_sap_ctas(qcd_ctx *c, int min_ctas) {
    int rc = ready(c);
    if (rc) return rc;
    if (min_ctas < -2 || min_ctas > 16) return fail(c, QCD_ERR_ARG, "min_ctas must lie in -2..16");
    QCD_CUDA(c, c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    c->sap_ctas_user = min_ctas;
    use_sap_ctas(c, 0);
    return QCD_OK;
}

int qcd_debug_inject_breakdown(qcd_ctx *c, int count) {
    int rc = ready(c);
    if (rc) return rc;
    if (count < 0) return fail(c, QCD_ERR_ARG, "count must be >= 0");
    c->inject_breakdown = count;
    return QCD_OK;
}

int qcd_debug_tc_skip_commit(qcd_ctx *c, int on) {
    int rc = ready(c);
    if (rc) return rc;
    c->tc_skip_commit = on != 0;
    return QCD_OK;
}

int qcd_set_sap_form(qcd_ctx *c, int form) {
    int rc = ready(c);
    if (rc) return rc;
    if (form < 0 || form > 2) return fail(c, QCD_ERR_ARG, "form must lie in 0..2");
    c->sap_form = form;
    return QCD_OK;
}

int qcd_sap_plan_tables(const int dims[4], const int block[4], const int subblock[4], int sap_ctas, int half, int sms,
                        int meta[8], int *level, int *owner, int *slot, int *chunk, unsigned char *flags) {
    if (!dims || !block || !subblock || !meta || sap_ctas < -2 || sap_ctas > 16 || sms < 1) return QCD_ERR_ARG;
    qcd_ctx c;  // host-side planning only: no device, stream or allocation is touched
    c.lat.V = 1;
    for (int m = 0; m < 4; m++) {
        if (dims[m] < 2) return QCD_ERR_ARG;
        c.lat.L[m] = dims[m];
        c.lat.V *= dims[m];
    }
    c.sms_override = sms;
    SapPlan p;
    if (sap_plan_host(&c, block, subblock, p, sap_ctas, half != 0) != QCD_OK) return QCD_ERR_ARG;
    const int vals[8] = {p.vol, p.nsteps, p.C, p.nchunks, p.nslot, p.slab_vol, p.tile ? 2 : p.thread ? 1 : 0,
                         (int)p.smem_bytes};
    for (int k = 0; k < 8; k++) meta[k] = vals[k];
    for (int st = 0; st < p.nsteps; st++)
        for (int k = p.h_step_ptr[st]; k < p.h_step_ptr[st + 1]; k++)
            if (level) level[p.h_step_site[k]] = st;
    for (int yl = 0; yl < p.vol; yl++) {
        if (owner) owner[yl] = (p.thread || p.tile) ? 0 : p.h_own[yl] >> 24;
        if (slot) slot[yl] = (p.thread || p.tile) ? yl : p.h_own[yl] & 0xffffff;
    }
    const int nct = (p.thread || p.tile) ? 1 : p.C;
    for (int r = 0; r < nct; r++)
        for (int ch = 0; ch < p.nchunks; ch++)
            for (int k = p.h_chunk_ptr[r * (p.nchunks + 1) + ch]; k < p.h_chunk_ptr[r * (p.nchunks + 1) + ch + 1]; k++)
                if (chunk) chunk[p.h_chunk_site[k]] = ch;
    if (flags)
        for (int k = 0; k < 2 * p.nchunks; k++) flags[k] = p.h_flags[k];
    return QCD_OK;
}

int qcd_set_profiling(qcd_ctx *c, int on) {
    int rc = ready(c);
    if (rc) return rc;
    if (!on && (rc = prof_collect(c))) return rc;
    c->prof.on = on != 0;
    return QCD_OK;
}

int qcd_kernel_stats(qcd_ctx *c, int kclass, long *launches, double *ms, int reset) {
    int rc = ready(c);
    if (rc) return rc;
    if (kclass < 0 || kclass >= QCD_K_COUNT) return fail(c, QCD_ERR_ARG, "kernel class out of range");
    if ((rc = prof_collect(c))) return rc;
    if (launches) *launches = c->prof.launches[kclass];
    if (ms) *ms = c->prof.ms[kclass];
    if (reset) {
        c->prof.launches[kclass] = 0;
        c->prof.ms[kclass] = 0;
    }
    return QCD_OK;
}

long qcd_launch_count(const qcd_ctx *c) { return c ? c->total_launches : 0; }

long qcd_learned_weight_count(void) { return learned_weight_count(); }

int qcd_learned_set_weights(qcd_ctx *c, const float *w, long n) {
    int rc = ready(c);
    if (rc) return rc;
    if (!c->have_gauge) return fail(c, QCD_ERR_STATE, "qcd_load_gauge must be called first");
    if (!w || n != learned_weight_count()) return fail(c, QCD_ERR_ARG, "weight count mismatch");
    if ((rc = learned_set_weights(c, (const float2 *)w, is_device_ptr(w)))) return rc;
    c->net.verdict = -1;
    QCD_CUDA(c, cudaStreamSynchronize(c->stream));
    return QCD_OK;
}

int qcd_learned_get_weights(qcd_ctx *c, float *w, long n) {
    int rc = ready(c);
    if (rc) return rc;
    if (!w || n != learned_weight_count()) return fail(c, QCD_ERR_ARG, "weight count mismatch");
    return learned_get_weights(c, (float2 *)w);
}

// Weights file: one JSON header line, then the complex64 weights (little-endian float pairs) in
// the layout of qcd_learned_set_weights.
static std::string learned_header(long n) {
    std::string ch;
    for (int l = 0; l <= kLearnedLayers; l++) ch += (l ? ", " : "") + std::to_string(kLearnedChans[l]);
    return "{\"format\": \"qcd-learned-weights\", \"version\": 1, \"layers\": " + std::to_string(kLearnedLayers) +
           ", \"channels\": [" + ch + "], \"layout\": \"[layer][9][cout][cin][4][4]\", \"dtype\": \"complex64\", "
           "\"count\": " + std::to_string(n) + "}";
}

int qcd_learned_save(const qcd_ctx *cc, const char *path) {
    qcd_ctx *c = const_cast<qcd_ctx *>(cc);  // reads the weights only
    int rc = ready(c);
    if (rc) return rc;
    if (!path) return fail(c, QCD_ERR_ARG, "path is NULL");
    if (!c->net.ready) return fail(c, QCD_ERR_STATE, "no learned weights (qcd_learned_set_weights first)");
    const long n = learned_weight_count();
    std::vector<float> w(2 * (size_t)n);
    if ((rc = learned_get_weights(c, (float2 *)w.data()))) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(c, QCD_ERR_ARG, std::string("cannot open ") + path + " for writing");
    const std::string head = learned_header(n) + "\n";
    const bool ok = std::fwrite(head.data(), 1, head.size(), f) == head.size() &&
                    std::fwrite(w.data(), sizeof(float), w.size(), f) == w.size();
    if (std::fclose(f) != 0 || !ok) return fail(c, QCD_ERR_ARG, std::string("cannot write ") + path);
    return QCD_OK;
}

int qcd_learned_load(qcd_ctx *c, const char *path) {
    int rc = ready(c);
    if (rc) return rc;
    if (!path) return fail(c, QCD_ERR_ARG, "path is NULL");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(c, QCD_ERR_ARG, std::string("cannot open ") + path);
    const long n = learned_weight_count();
    const std::string want = learned_header(n);
    std::string line;
    for (int ch; (ch = std::fgetc(f)) != EOF && ch != '\n' && line.size() < 4096;) line.push_back((char)ch);
    std::vector<float> w(2 * (size_t)n);
    const bool ok = line == want && std::fread(w.data(), sizeof(float), w.size(), f) == w.size() &&
                    std::fgetc(f) == EOF;
    std::fclose(f);
    if (!ok) return fail(c, QCD_ERR_ARG, std::string(path) + ": not a weights file of this network (" + want + ")");
    return qcd_learned_set_weights(c, w.data(), n);
}

// stage a complex64 [k][V][12] field (host or device) into the internal plane layout
static int stage_in32(qcd_ctx *c, float4 *dst, const float *src, int k, char *scratch) {
    const size_t bytes = 8 * 12 * (size_t)c->lat.V * k;
    const void *s = src;
    if (!is_device_ptr(src)) {
        QCD_CUDA(c, cudaMemcpyAsync(scratch, src, bytes, cudaMemcpyHostToDevice, c->stream));
        s = scratch;
    }
    return spinor32_to_internal(c, dst, (const float2 *)s, k);
}

int qcd_learned_apply(qcd_ctx *c, float *out, const float *in) {
    int rc = ready(c);
    if (rc) return rc;
    if (!c->net.ready) return fail(c, QCD_ERR_STATE, "qcd_learned_set_weights must be called first");
    if (!out || !in) return fail(c, QCD_ERR_ARG, "NULL argument");
    const size_t bytes = 8 * 12 * (size_t)c->lat.V;
    if ((rc = ensure_io(c, 3 * bytes))) return rc;
    char *io = (char *)c->d_io;
    float4 *x = (float4 *)io, *y = (float4 *)(io + bytes);
    if ((rc = stage_in32(c, x, in, 1, io + 2 * bytes))) return rc;
    if ((rc = learned_forward(c, y, x))) return rc;
    const bool dev_out = is_device_ptr(out);
    if ((rc = spinor32_from_internal(c, (float2 *)(dev_out ? (char *)out : io + 2 * bytes), y, 1))) return rc;
    if (!dev_out) QCD_CUDA(c, cudaMemcpyAsync(out, io + 2 * bytes, bytes, cudaMemcpyDeviceToHost, c->stream));
    return learned_tc_status(c);  // synchronises
}

int qcd_learned_loss_grad(qcd_ctx *c, const float *rho, const float *eps, double *loss, float *grad) {
    int rc = ready(c);
    if (rc) return rc;
    if (!c->net.ready) return fail(c, QCD_ERR_STATE, "qcd_learned_set_weights must be called first");
    if (!rho || !eps) return fail(c, QCD_ERR_ARG, "NULL argument");
    const size_t bytes = 8 * 12 * (size_t)c->lat.V;
    if ((rc = ensure_io(c, 5 * bytes))) return rc;
    char *io = (char *)c->d_io;
    float4 *r = (float4 *)io, *e4 = (float4 *)(io + bytes), *y = (float4 *)(io + 2 * bytes);
    float2 *es = (float2 *)(io + 3 * bytes);
    if ((rc = stage_in32(c, r, rho, 1, io + 4 * bytes))) return rc;
    if ((rc = stage_in32(c, e4, eps, 1, io + 4 * bytes))) return rc;
    if ((rc = plane_to_site(c, es, e4))) return rc;
    if ((rc = learned_zero_grad(c))) return rc;
    double l = 0;
    if ((rc = learned_loss_grad(c, r, es, &l, y))) return rc;
    if (loss) *loss = l;
    if (grad)
        QCD_CUDA(c, cudaMemcpyAsync(grad, c->net.grad, sizeof(float2) * learned_weight_count(),
                                    cudaMemcpyDeviceToHost, c->stream));
    return learned_tc_status(c);  // synchronises
}

int qcd_learned_train(qcd_ctx *c, const float *sources, int npairs, const qcd_params *p, int epochs, int batch,
                      float lr, double *history) {
    int rc = ready(c);
    if (rc) return rc;
    if ((rc = need_clover(c))) return rc;
    if (!c->net.ready) return fail(c, QCD_ERR_STATE, "qcd_learned_set_weights must be called first");
    if (!sources || npairs < 1 || epochs < 0 || batch < 1 || !(lr > 0)) return fail(c, QCD_ERR_ARG, "bad training arguments");
    qcd_params pp = *p;
    pp.learned = 0;  // the pairs measure the error of plain SAP
    c->net.verdict = -1;
    if ((rc = check_params(c, &pp))) return rc;
    if (pp.block_solver != 0) return fail(c, QCD_ERR_ARG, "training pairs come from the SSOR block solver (block_solver 0)");
    if ((rc = sap_prepare(c, pp.block, pp.subblock, pp.sap_storage == QCD_F16))) return rc;
    const long V = c->lat.V;
    const size_t f32 = 96 * (size_t)V, f64 = 192 * (size_t)V;
    // pairs: rho (plane FP32) then eps (site FP32), per pair
    const size_t need = 2 * f32 * (size_t)npairs;
    if (c->net.pairs_bytes < need) {
        dev_free(c, c->net.pairs);
        c->net.pairs = nullptr;
        c->net.pairs_bytes = 0;
        if ((rc = dev_alloc(c, (void **)&c->net.pairs, need))) return rc;
        c->net.pairs_bytes = need;
    }
    char *pairs = (char *)c->net.pairs;
    const int chunk = npairs < 16 ? npairs : 16;
    // chunk buffers: staging, r, x, Dx, SAP work (2), FP64 rhs and solution
    void *tmpb = nullptr;
    if ((rc = dev_alloc(c, &tmpb, (size_t)chunk * (6 * f32 + 2 * f64)))) return rc;
    struct Free {
        qcd_ctx *c;
        void *p;
        ~Free() { dev_free(c, p); }
    } guard{c, tmpb};
    char *tb = (char *)tmpb;
    char *stg = tb;
    float4 *r = (float4 *)(tb + chunk * f32), *x = (float4 *)(tb + 2 * chunk * f32);
    float4 *dx = (float4 *)(tb + 3 * chunk * f32), *work = (float4 *)(tb + 4 * chunk * f32);
    double2 *b64 = (double2 *)(tb + 6 * chunk * f32), *x64 = (double2 *)(tb + 6 * chunk * f32 + chunk * f64);
    qcd_params ps = pp;
    ps.tol = 1e-9;
    const bool dev_src = is_device_ptr(sources);
    for (int k0 = 0; k0 < npairs; k0 += chunk) {
        const int k = std::min(chunk, npairs - k0);
        const float *src = sources + (size_t)k0 * 24 * V;
        if (!dev_src) {
            QCD_CUDA(c, cudaMemcpyAsync(stg, src, (size_t)k * f32, cudaMemcpyHostToDevice, c->stream));
            src = (const float *)stg;
        }
        if ((rc = spinor32_to_internal(c, r, (const float2 *)src, k))) return rc;
        if ((rc = sap_apply(c, x, r, work, pp.omega, pp.nsweep, pp.nsap, k))) return rc;
        if ((rc = dslash32(c, dx, x, k))) return rc;
        if ((rc = sub_plane(c, dx, r, dx, k))) return rc;  // rho = r - D M_SAP r
        for (int j = 0; j < k; j++)
            QCD_CUDA(c, cudaMemcpyAsync(pairs + (size_t)(k0 + j) * 2 * f32, (char *)dx + j * f32, f32,
                                        cudaMemcpyDeviceToDevice, c->stream));
        // eps = D^{-1} rho in FP64
        if ((rc = spinor32_to_64(c, b64, dx, k))) return rc;
        QCD_CUDA(c, cudaMemsetAsync(x64, 0, (size_t)k * f64, c->stream));
        qcd_stats st;
        std::memset(&st, 0, sizeof(st));
        int s = solve(c, x64, b64, &ps, k, &st);
        if (s != QCD_OK) return s == QCD_ERR_NOCONV || s == QCD_ERR_BREAKDOWN ? fail(c, s, "training pairs: solve failed") : s;
        if ((rc = spinor64_to_32(c, x, x64, k))) return rc;
        for (int j = 0; j < k; j++)
            if ((rc = plane_to_site(c, (float2 *)(pairs + (size_t)(k0 + j) * 2 * f32 + f32), x + j * 6 * V))) return rc;
    }
    // training
    float4 *ybuf = dx;
    auto pair_loss = [&](int k, bool grad, double *l) -> int {
        const float4 *rho = (const float4 *)(pairs + (size_t)k * 2 * f32);
        const float2 *eps = (const float2 *)(pairs + (size_t)k * 2 * f32 + f32);
        if (!grad) QCD_CUDA(c, cudaMemsetAsync(c->net.grad, 0, sizeof(float2) * learned_weight_count(), c->stream));
        return learned_loss_grad(c, rho, eps, l, ybuf);
    };
    double total = 0;
    for (int k = 0; k < npairs; k++) {
        double l = 0;
        if ((rc = pair_loss(k, false, &l))) return rc;
        total += l;
    }
    if (history) history[0] = total / npairs;
    for (int e = 0; e < epochs; e++) {
        total = 0;
        for (int b0 = 0; b0 < npairs; b0 += batch) {
            if ((rc = learned_zero_grad(c))) return rc;
            for (int k = b0; k < std::min(npairs, b0 + batch); k++) {
                double l = 0;
                if ((rc = pair_loss(k, true, &l))) return rc;
                total += l;
            }
            if ((rc = learned_adam(c, lr))) return rc;
        }
        if (history) history[e + 1] = total / npairs;
    }
    return learned_tc_status(c);  // synchronises
}

int qcd_learned_evaluate(qcd_ctx *c, const double *b, int nrhs, const qcd_params *p, qcd_learned_verdict *out) {
    int rc = ready(c);
    if (rc) return rc;
    if ((rc = need_clover(c))) return rc;
    if (!c->net.ready) return fail(c, QCD_ERR_STATE, "qcd_learned_set_weights must be called first");
    if (!b || nrhs < 1 || !p) return fail(c, QCD_ERR_ARG, "qcd_learned_evaluate: bad b, nrhs or params");
    const size_t bytes = 16 * 12 * (size_t)c->lat.V * nrhs;
    void *xb = nullptr;
    if ((rc = dev_alloc(c, &xb, bytes))) return rc;
    struct Free {
        qcd_ctx *c;
        void *p;
        ~Free() { dev_free(c, p); }
    } guard{c, xb};
    qcd_learned_verdict v;
    std::memset(&v, 0, sizeof(v));
    // each variant: one warm solve, then the timed one
    auto run = [&](int learned, double *ms, double *relres, int *outer, int *inner) -> int {
        qcd_params q = *p;
        q.learned = learned;
        qcd_stats st;
        for (int k = 0; k < 2; k++) {
            QCD_CUDA(c, cudaMemsetAsync(xb, 0, bytes, c->stream));
            std::memset(&st, 0, sizeof(st));
            const int s = qcd_solve(c, (double *)xb, b, &q, nrhs, &st);
            if (s != QCD_OK && s != QCD_ERR_NOCONV && s != QCD_ERR_BREAKDOWN) return s;
            if (s != QCD_OK) st.true_rel_res = st.true_rel_res > 0 ? st.true_rel_res : 1.0;
        }
        *ms = st.ms_total;
        *relres = st.true_rel_res;
        *outer = st.outer_iters;
        *inner = st.inner_iters;
        return QCD_OK;
    };
    if ((rc = run(0, &v.plain_ms, &v.plain_relres, &v.plain_outer, &v.plain_inner))) return rc;
    if ((rc = run(2, &v.learned_ms, &v.learned_relres, &v.learned_outer, &v.learned_inner))) return rc;
    v.use_learned = (v.learned_relres <= p->tol && v.learned_ms < v.plain_ms) ? 1 : 0;
    c->net.verdict = v.use_learned;
    c->err.clear();
    if (out) *out = v;
    return QCD_OK;
}

int qcd_bench_dslash(qcd_ctx *c, int prec, int nrhs, int iters) {
    int rc = ready(c);
    if (rc) return rc;
    if ((rc = need_clover(c))) return rc;
    if ((prec != QCD_F64 && prec != QCD_F32 && prec != QCD_F16 && prec != QCD_F32_SU3 && prec != QCD_F32X2) ||
        nrhs < 1 || iters < 1)
        return fail(c, QCD_ERR_ARG, "qcd_bench_dslash: bad precision, nrhs or iters");
    const size_t bytes = (prec == QCD_F64 || prec == QCD_F32X2 ? 16 : 8) * 12 * c->lat.V * (size_t)nrhs;
    if (c->bench_bytes < bytes) {
        dev_free(c, c->bench_in);
        dev_free(c, c->bench_out);
        c->bench_in = c->bench_out = nullptr;
        c->bench_bytes = 0;
        if ((rc = dev_alloc(c, &c->bench_in, bytes))) return rc;
        if ((rc = dev_alloc(c, &c->bench_out, bytes))) return rc;
        c->bench_bytes = bytes;
        // a deterministic non-trivial input: constant bytes
        QCD_CUDA(c, cudaMemsetAsync(c->bench_in, 0x3c, bytes, c->stream));
    }
    for (int i = 0; i < iters; i++) {
        if (prec == QCD_F64) rc = dslash64(c, (double2 *)c->bench_out, (const double2 *)c->bench_in, nrhs);
        else if (prec == QCD_F32X2) rc = dslash_x2(c, (double2 *)c->bench_out, (const float4 *)c->bench_in, nrhs);
        else if (prec == QCD_F16) rc = dslash16(c, (float4 *)c->bench_out, (const float4 *)c->bench_in, nrhs);
        else if (prec == QCD_F32_SU3) rc = dslash12(c, (float4 *)c->bench_out, (const float4 *)c->bench_in, nrhs);
        else rc = dslash32(c, (float4 *)c->bench_out, (const float4 *)c->bench_in, nrhs);
        if (rc) return rc;
    }
    return QCD_OK;
}

}  // extern "C"
