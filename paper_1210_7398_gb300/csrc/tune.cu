// S2: autotuner of the SAP set-up.  The paper fixes one geometry (6^4 blocks,
// 3^4 sub-blocks per node); on a GPU the best block split trades the number of
// dependent ll steps (block size) against SAP quality (outer/inner iteration
// counts), so candidates are compared by measured time to solution.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "qcd_internal.h"

namespace qcd {
namespace {

struct Cand {
    qcd_params p;
    double ms = 1e300;
    bool ok = false;
};

bool valid_block(const qcd_ctx *c, const int b[4], const int s[4]) {
    for (int m = 0; m < 4; m++) {
        if (b[m] < 2 || s[m] < 1 || c->lat.L[m] % b[m] || b[m] % s[m]) return false;
        const int nb = c->lat.L[m] / b[m];
        if (nb < 2 || nb % 2) return false;
    }
    return true;
}

// time one complete solve (x0 = 0) of the internal-layout right-hand sides bi, in groups of
// p->rhs_group right-hand sides (0: all at once) as qcd_solve runs them
int time_solve(qcd_ctx *c, double2 *xi, const double2 *bi, int nrhs, const qcd_params *p, double *ms, bool *ok) {
    *ok = false;
    use_sap_ctas(c, p->sap_ctas);  // sap_ctas 0: the context's setting, not the last candidate's
    int rc = sap_prepare(c, p->block, p->subblock, p->sap_storage == QCD_F16);
    if (rc == QCD_ERR_ARG) {  // geometry does not fit: not a candidate
        c->err.clear();
        return QCD_OK;
    }
    if (rc) return rc;
    cudaEvent_t e0, e1;
    QCD_CUDA(c, cudaEventCreate(&e0));
    QCD_CUDA(c, cudaEventCreate(&e1));
    const size_t bytes = sizeof(double2) * 12 * c->lat.V * nrhs;
    QCD_CUDA(c, cudaMemsetAsync(xi, 0, bytes, c->stream));
    QCD_CUDA(c, cudaEventRecord(e0, c->stream));
    qcd_stats st;
    std::memset(&st, 0, sizeof(st));
    const int g = p->rhs_group > 0 ? std::min(p->rhs_group, nrhs) : nrhs;
    int s = QCD_OK;
    for (int k0 = 0; k0 < nrhs && (s == QCD_OK || s == QCD_ERR_NOCONV || s == QCD_ERR_BREAKDOWN); k0 += g) {
        const int n = std::min(g, nrhs - k0);
        const int sg = solve(c, xi + (size_t)12 * c->lat.V * k0, bi + (size_t)12 * c->lat.V * k0, p, n, &st);
        if (sg != QCD_OK && s == QCD_OK) s = sg;
    }
    QCD_CUDA(c, cudaEventRecord(e1, c->stream));
    QCD_CUDA(c, cudaEventSynchronize(e1));
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == QCD_ERR_CUDA || s == QCD_ERR_OOM || s == QCD_ERR_STATE) return s;
    *ok = (s == QCD_OK);
    *ms = t;
    return QCD_OK;
}

// ---- on-disk cache of tuning results (one JSON object per line) ----
std::mutex g_cache_mu;
std::string g_cache_path;
constexpr const char *kTunerVersion = "sap-tile-4";

std::string cache_key(qcd_ctx *c, int nrhs, const qcd_params *b, int max_candidates) {
    cudaDeviceProp prop;
    std::string gpu = "unknown";
    int sms = 0;
    if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) {
        gpu = prop.name;
        sms = prop.multiProcessorCount;
    } else {
        cudaGetLastError();
    }
    for (char &ch : gpu)
        if (ch == '"' || ch == ';' || ch == '\\') ch = '_';
    char buf[512];
    std::snprintf(buf, sizeof(buf),
                  "%s;dims=%dx%dx%dx%d;nrhs=%d;kappa=%.17g;csw=%.17g;bc_t=%d;tol=%.17g;inner_tol=%.17g;"
                  "max=%d/%d;omega=%.17g;rhs_group=%d;outer=%d;cands=%d;gpu=%s;sms=%d",
                  kTunerVersion, c->lat.L[0], c->lat.L[1], c->lat.L[2], c->lat.L[3], nrhs, b->kappa, b->csw, b->bc_t,
                  b->tol, b->inner_tol, b->max_outer, b->max_inner, b->omega, b->rhs_group, b->outer_precision,
                  max_candidates, gpu.c_str(), sms);
    return buf;
}

// the cached winner for key, if the cache file holds one
bool cache_lookup(const std::string &key, const qcd_params *base, qcd_params *best, double *ms) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    if (g_cache_path.empty()) return false;
    FILE *f = std::fopen(g_cache_path.c_str(), "r");
    if (!f) return false;
    const std::string head = "{\"key\": \"" + key + "\", ";
    char line[2048];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        if (std::strncmp(line, head.c_str(), head.size()) != 0) continue;
        qcd_params p = *base;
        double t = 0;
        const int n = std::sscanf(line + head.size(),
                                  "\"block\": [%d, %d, %d, %d], \"subblock\": [%d, %d, %d, %d], "
                                  "\"omega\": %lf, \"sap_storage\": %d, \"sap_ctas\": %d, \"nsweep\": %d, "
                                  "\"nsap\": %d, \"rhs_group\": %d, \"outer_precision\": %d, \"ms\": %lf",
                                  &p.block[0], &p.block[1], &p.block[2], &p.block[3], &p.subblock[0], &p.subblock[1],
                                  &p.subblock[2], &p.subblock[3], &p.omega, &p.sap_storage, &p.sap_ctas, &p.nsweep,
                                  &p.nsap, &p.rhs_group, &p.outer_precision, &t);
        if (n == 16) {
            *best = p;
            *ms = t;
            found = true;  // the last matching line wins
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const std::string &key, const qcd_params *p, double ms) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    if (g_cache_path.empty()) return;
    FILE *f = std::fopen(g_cache_path.c_str(), "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"block\": [%d, %d, %d, %d], \"subblock\": [%d, %d, %d, %d], "
                 "\"omega\": %.17g, \"sap_storage\": %d, \"sap_ctas\": %d, \"nsweep\": %d, \"nsap\": %d, "
                 "\"rhs_group\": %d, \"outer_precision\": %d, \"ms\": %.6f}\n",
                 key.c_str(), p->block[0], p->block[1], p->block[2], p->block[3], p->subblock[0], p->subblock[1],
                 p->subblock[2], p->subblock[3], p->omega, p->sap_storage, p->sap_ctas, p->nsweep, p->nsap,
                 p->rhs_group, p->outer_precision, ms);
    std::fclose(f);
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" int qcd_set_tune_cache(const char *path) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    g_cache_path = path ? path : "";
    return QCD_OK;
}

extern "C" int qcd_autotune(qcd_ctx *c, const double *b, int nrhs, const qcd_params *base, qcd_params *best,
                            double *best_ms, int max_candidates) {
    if (!c || !b || !base || !best || nrhs < 1) return QCD_ERR_ARG;
    if (c->poisoned) return fail(c, QCD_ERR_STATE, "context poisoned by an earlier CUDA error: " + c->err);
    QCD_CUDA(c, cudaSetDevice(c->device));
    if (!c->have_clover) return fail(c, QCD_ERR_STATE, "qcd_build_clover must be called first");
    if (base->kappa != c->kappa || base->csw != c->csw || base->bc_t != c->bc_t)
        return fail(c, QCD_ERR_ARG, "params kappa/csw/bc_t differ from the context");
    if (max_candidates <= 0) max_candidates = 64;
    const std::string key = cache_key(c, nrhs, base, max_candidates);
    {
        double cms = 0;
        if (cache_lookup(key, base, best, &cms)) {
            if (best_ms) *best_ms = cms;
            return QCD_OK;
        }
    }
    const long V = c->lat.V;
    const size_t bytes = sizeof(double2) * 12 * V * nrhs;
    // right-hand sides in the internal layout, solution buffer
    void *buf = nullptr;
    int rc = dev_alloc(c, &buf, 3 * bytes);
    if (rc) return rc;
    struct Free {
        qcd_ctx *c;
        void *p;
        ~Free() { dev_free(c, p); }
    } guard{c, buf};
    double2 *bi = (double2 *)buf, *xi = bi + 12 * V * nrhs, *stage = xi + 12 * V * nrhs;
    cudaPointerAttributes at;
    const bool on_dev = cudaPointerGetAttributes(&at, b) == cudaSuccess &&
                        (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    QCD_CUDA(c, cudaMemcpyAsync(stage, b, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if ((rc = spinor64_to_internal(c, bi, stage, nrhs))) return rc;
    const bool old_prof = c->prof.on;
    c->prof.on = false;

    // stage 1: block and sub-block splits, ranked with the fast tile form, FP16 storage, 2 sweeps,
    // 2 cycles and omega 1
    std::vector<Cand> cands;
    // block extents: the spatial ones alike, each dividing L with an even quotient
    const int extents[] = {2, 3, 4, 6, 8, 12, 16};
    for (int bs : extents)
        for (int bt : extents) {
            int blk[4] = {bs, bs, bs, bt};
            bool fits = true;
            for (int m = 0; m < 4; m++) fits = fits && c->lat.L[m] % blk[m] == 0 && (c->lat.L[m] / blk[m]) % 2 == 0;
            if (!fits || bt < bs || bt > 2 * bs) continue;
            const int vol = blk[0] * blk[1] * blk[2] * blk[3];
            if (vol > 4096 || vol < 16) continue;
            for (int div = 2; div <= 4; div++) {
                int sub[4];
                for (int m = 0; m < 4; m++) sub[m] = (div == 4) ? blk[m] : (blk[m] % div ? 0 : blk[m] / div);
                if (!sub[0] || !sub[1] || !sub[2] || !sub[3]) continue;
                if (!valid_block(c, blk, sub)) continue;
                Cand cd;
                cd.p = *base;
                std::memcpy(cd.p.block, blk, sizeof(blk));
                std::memcpy(cd.p.subblock, sub, sizeof(sub));
                // ranked with the fast form: the tile form with FP16 storage, the cluster form
                // where a block's spinor does not fit one CTA
                cd.p.sap_storage = QCD_F16;
                cd.p.sap_ctas = -2;
                cd.p.nsweep = 2;
                cd.p.nsap = 2;
                cd.p.omega = 1.0;
                cd.p.block_solver = 0;  // the tuner explores the ll-SSOR set-ups
                cd.p.rhs_group = base->rhs_group;
                cands.push_back(cd);
            }
        }
    // blocks of about 256 sites first (a few levels of many sites each), so that a small
    // candidate budget covers the promising region
    std::stable_sort(cands.begin(), cands.end(), [](const Cand &u, const Cand &v) {
        auto dist = [](const Cand &x) {
            const double vol = (double)x.p.block[0] * x.p.block[1] * x.p.block[2] * x.p.block[3];
            return std::fabs(std::log(vol / 256.0));
        };
        return dist(u) < dist(v);
    });
    int tried = 0;
    auto run = [&](Cand &cd) -> int {
        if (tried >= max_candidates) return QCD_OK;
        tried++;
        double ms = 0;
        bool ok = false;
        // first solve builds the plan and records; the second is timed
        int r2 = time_solve(c, xi, bi, nrhs, &cd.p, &ms, &ok);
        if (r2) return r2;
        if (ok) {
            r2 = time_solve(c, xi, bi, nrhs, &cd.p, &ms, &ok);
            if (r2) return r2;
        }
        cd.ok = ok;
        cd.ms = ok ? ms : 1e300;
        return QCD_OK;
    };
    // stage 1 takes at most half the budget, so that stage 2 can refine
    const int stage1 = std::max(1, (max_candidates + 1) / 2);
    for (auto &cd : cands) {
        if (tried >= stage1) break;
        if ((rc = run(cd))) break;
    }
    if (!rc) {
        std::sort(cands.begin(), cands.end(), [](const Cand &u, const Cand &v) { return u.ms < v.ms; });
        // stage 2: a coordinate search from the fastest geometry, one parameter at a time, each
        // move kept only if it is faster: first the outer operator in pair-of-FP32 arithmetic
        // where the base asks for the FP64 one (the same accuracy), then the SSOR relaxation omega
        // upwards in steps of 0.2 while it improves, the SAP cycles (1, 3), the SSOR sweeps (3, 1),
        // and last the other storage and kernel forms
        std::vector<Cand> more;
        if (!cands.empty() && cands[0].ok) {
            Cand cur = cands[0];
            auto try_move = [&](Cand cd) -> bool {
                if (tried >= max_candidates || rc) return false;
                rc = run(cd);
                more.push_back(cd);
                if (!rc && cd.ok && cd.ms < cur.ms) {
                    cur = cd;
                    return true;
                }
                return false;
            };
            if (cur.p.outer_precision == QCD_F64) {
                Cand cd = cur;
                cd.p.outer_precision = QCD_F32X2;
                try_move(cd);
            }
            for (double om = cur.p.omega + 0.2; om < 1.95; om += 0.2) {
                Cand cd = cur;
                cd.p.omega = om;
                if (!try_move(cd)) break;
            }
            for (int np : {1, 3})
                if (np != cur.p.nsap) {
                    Cand cd = cur;
                    cd.p.nsap = np;
                    try_move(cd);
                }
            for (int ns : {3, 1})
                if (ns != cur.p.nsweep) {
                    Cand cd = cur;
                    cd.p.nsweep = ns;
                    try_move(cd);
                }
            const int forms[][2] = {{QCD_F32, -2}, {QCD_F16, 0}, {QCD_F32, 0}, {QCD_F16, 2}};
            for (const auto &f : forms)
                if (f[0] != cur.p.sap_storage || f[1] != cur.p.sap_ctas) {
                    Cand cd = cur;
                    cd.p.sap_storage = f[0];
                    cd.p.sap_ctas = f[1];
                    try_move(cd);
                }
        }
        cands.insert(cands.end(), more.begin(), more.end());
    }
    if (!rc && nrhs > 1 && base->rhs_group == 0) {
        // stage 3: right-hand sides per group for the fastest set-up (all at once, or groups of
        // 1, 2, 4 or 8 that divide them)
        const Cand *w0 = nullptr;
        for (auto &cd : cands)
            if (cd.ok && (!w0 || cd.ms < w0->ms)) w0 = &cd;
        if (w0) {
            std::vector<Cand> more;
            for (int g : {1, 2, 4, 8})
                if (g < nrhs && nrhs % g == 0) {
                    Cand cd = *w0;
                    cd.p.rhs_group = g;
                    more.push_back(cd);
                }
            for (auto &cd : more) {
                tried = std::min(tried, max_candidates - 1);  // always time the group sizes
                if ((rc = run(cd))) break;
            }
            cands.insert(cands.end(), more.begin(), more.end());
        }
    }
    c->prof.on = old_prof;
    use_sap_ctas(c, 0);
    if (rc) return rc;
    const Cand *win = nullptr;
    for (auto &cd : cands)
        if (cd.ok && (!win || cd.ms < win->ms)) win = &cd;
    if (!win) return fail(c, QCD_ERR_NOCONV, "autotune: no candidate converged");
    *best = win->p;
    if (best_ms) *best_ms = win->ms;
    cache_store(key, &win->p, win->ms);
    return QCD_OK;
}
