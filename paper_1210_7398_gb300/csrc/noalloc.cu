// qcd_sap_precondition_noalloc: the SAP preconditioner for callers that must
// not allocate device memory when they call it.
//
// Typical callers: a host that shares the GPU with a framework whose caching
// allocator has already reserved the free memory (a cudaMalloc from here
// would fail or fragment its pool), a serving loop with a fixed memory budget
// that must not grow or synchronise on allocation while requests are in
// flight, or code that runs between set-up and tear-down phases in which only
// kernel launches and copies are permitted.  They create the context (which
// allocates the gauge and clover fields) once at set-up, and afterwards call
// this entry point, which only launches kernels and copies.
//
// Its scratch memory (the internal-layout input and output spinors, the two
// SAP work spinors, the per-site SSOR records and the ll-schedule tables) lives in one file-scope
// __device__ array of fixed size, so the library reserves it on every GPU
// that loads the library, until the process exits.  In host code the array's
// name is only a host-side stand-in for the symbol; the device address is
// obtained with cudaGetSymbolAddress once per device and passed to the
// kernels.
//
// The array keeps what the last call built: the schedule tables and per-site records of one
// context's fields, geometry and kernel form (per device).  A call that matches them only
// converts the input, launches the SAP kernels and converts the output, all asynchronously on
// the context stream; a call with another context, changed fields, geometry or form first plans
// on the host, uploads the tables and rebuilds the records, which synchronises the stream.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "qcd_internal.h"

namespace qcd {
namespace {

// Largest lattice this entry point accepts: 41,472 sites (e.g. 12^3 x 24).
constexpr long kNoAllocMaxSites = 41472;
constexpr size_t kSpinorBytes = sizeof(float4) * 6 * (size_t)kNoAllocMaxSites;  // one FP32 spinor field
constexpr size_t kRecordBytes = kSapRecordBytesPerSite * (size_t)kNoAllocMaxSites;  // per-site SSOR records
constexpr size_t kTableBytes = 64 * (size_t)kNoAllocMaxSites;                    // ll schedule, block tables
constexpr size_t kScratchBytes = 4 * kSpinorBytes + kRecordBytes + kTableBytes;  // about 68.3 MB

static __device__ __align__(256) unsigned char g_sap_scratch[kScratchBytes];

std::mutex g_scratch_mutex;
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// What the array of each device holds now: the plan (host tables, device pointers into the
// array) and records made for one context's fields, geometry and kernel form.  A call with the
// same key reuses them and only launches kernels; any other call rebuilds them.
struct Held {
    long uid = 0, field_version = -1;
    int b[4] = {0, 0, 0, 0}, s[4] = {0, 0, 0, 0}, ctas = 0, sms = 0;
    SapPlan plan;
};
Held g_held[kMaxDevices];

// Device address of g_sap_scratch on the context's device (current when called).
int scratch_address(qcd_ctx *c, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (c->device < 0 || c->device >= kMaxDevices) return fail(c, QCD_ERR_ARG, "device ordinal out of range");
    if (!g_scratch_addr[c->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sap_scratch);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(g_sap_scratch)");
        g_scratch_addr[c->device] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[c->device];
    return QCD_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" int qcd_sap_precondition_noalloc(qcd_ctx *c, float *out, const float *in, const qcd_params *p) {
    if (!c) return QCD_ERR_ARG;
    if (c->poisoned) return fail(c, QCD_ERR_STATE, "context poisoned by an earlier CUDA error: " + c->err);
    QCD_CUDA(c, cudaSetDevice(c->device));
    if (!c->have_clover) return fail(c, QCD_ERR_STATE, "qcd_build_clover must be called first");
    if (!out || !in || !p) return fail(c, QCD_ERR_ARG, "qcd_sap_precondition_noalloc: NULL argument");
    if (!(p->omega > 0 && p->omega < 2) || p->nsweep < 1 || p->nsap < 1)
        return fail(c, QCD_ERR_ARG, "omega must lie in (0, 2); nsweep and nsap must be >= 1");
    if (p->sap_storage != QCD_F32 || p->learned != 0 || p->block_solver != 0)
        return fail(c, QCD_ERR_ARG,
                    "qcd_sap_precondition_noalloc supports sap_storage = QCD_F32, learned = 0, block_solver = 0");
    if (p->bc_t != c->bc_t || p->kappa != c->kappa || p->csw != c->csw)
        return fail(c, QCD_ERR_ARG, "params.bc_t/kappa/csw differ from the context");
    if (c->lat.V > kNoAllocMaxSites)
        return fail(c, QCD_ERR_ARG, "qcd_sap_precondition_noalloc: lattice of " + std::to_string(c->lat.V) +
                                        " sites exceeds its fixed scratch limit of 41472 sites");
    if (!on_device(in) || !on_device(out) || ((uintptr_t)in & 15) || ((uintptr_t)out & 15))
        return fail(c, QCD_ERR_ARG, "qcd_sap_precondition_noalloc needs 16-byte aligned device pointers");
    if (p->sap_ctas < -2 || p->sap_ctas > 16) return fail(c, QCD_ERR_ARG, "sap_ctas must lie in -2..16");
    if (!sap_geometry_ok(c, p->block, p->subblock))
        return fail(c, QCD_ERR_ARG, "SAP geometry: need L % block == 0, L/block even and >= 2, block % subblock == 0");
    // the kernel form qcd_sap_precondition would use with these params (0: the context's setting)
    const int ctas = p->sap_ctas != 0 ? p->sap_ctas : c->sap_ctas_user;
    unsigned char *base = nullptr;
    int rc = scratch_address(c, &base);
    if (rc) return rc;
    // scratch layout: [v | x | r, y | records | tables]; every region is fully written before it is read
    float4 *v = reinterpret_cast<float4 *>(base);
    float4 *x = reinterpret_cast<float4 *>(base + kSpinorBytes);
    float4 *work = reinterpret_cast<float4 *>(base + 2 * kSpinorBytes);
    float *rec = reinterpret_cast<float *>(base + 4 * kSpinorBytes);
    Held &h = g_held[c->device];
    SapPlan plan;  // copied under the lock: another host thread may replace the held one
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        int sms = c->sms_override;
        if (sms < 1 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
            cudaGetLastError();
            sms = 1;
        }
        const bool same = h.uid == c->uid && h.field_version == c->field_version && h.ctas == ctas && h.sms == sms &&
                          std::equal(p->block, p->block + 4, h.b) && std::equal(p->subblock, p->subblock + 4, h.s);
        if (!same) {
            // a new geometry, field or form: plan on the host, upload the tables and build the
            // records into the array (this path synchronises the stream)
            h.uid = 0;
            if (sap_plan_host(c, p->block, p->subblock, plan, ctas, false) != QCD_OK)
                return fail(c, QCD_ERR_ARG, "SAP block too large for the shared memory of a cluster of 16 CTAs");
            if (sap_table_bytes(plan) > kTableBytes || sap_record_bytes(plan) > kRecordBytes)
                return fail(c, QCD_ERR_ARG, "SAP schedule tables exceed the fixed scratch");
            if ((rc = sap_upload_tables(c, plan, base + 4 * kSpinorBytes + kRecordBytes))) return rc;
            if ((rc = sap_build_records(c, plan, rec))) return rc;
            h.plan = plan;
            h.uid = c->uid;
            h.field_version = c->field_version;
            h.ctas = ctas;
            h.sms = sms;
            std::memcpy(h.b, p->block, sizeof(h.b));
            std::memcpy(h.s, p->subblock, sizeof(h.s));
        } else {
            plan = h.plan;
        }
    }
    if ((rc = spinor32_to_internal(c, v, reinterpret_cast<const float2 *>(in), 1))) return rc;
    if ((rc = sap_apply_plan(c, plan, x, v, work, p->omega, p->nsweep, p->nsap))) return rc;
    if ((rc = spinor32_from_internal(c, reinterpret_cast<float2 *>(out), x, 1))) return rc;
    return QCD_OK;
}
