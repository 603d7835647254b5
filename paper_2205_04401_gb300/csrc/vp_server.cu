// Serving loop with continuous batching.
//
// A worker thread owns a set of CUDA streams ("slots").  Requests (a resident
// near-field build and 1..256 host densities) wait in a FIFO queue and are
// admitted as soon as a slot is free and their device footprint (densities,
// output, workspace) fits the HBM budget; each admitted request copies its
// densities in, runs the evaluation on its slot's stream and copies the
// result out, so the work of requests that arrive while others run overlaps
// on the device.  Completions are detected with CUDA events and free their
// slot and memory at once.  Meshes registered "cold" (host arrays only) are
// uploaded and their near field built on first use; the build time is part
// of that request's latency.  Every request runs exactly the kernels of
// vp_potential_eval, so its result does not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vp_internal.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Req {
    int64_t key = 0;
    const double* f_host = nullptr;
    double* u_host = nullptr;
    int d = 0;
    int state = RQ_QUEUED;
    int status = VP_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int slot = -1;
    void* dmem = nullptr;        // f, u and workspace in one stream-ordered allocation
    int64_t bytes = 0;
    cudaEvent_t ev = nullptr;
    int64_t evals = 0;
};

struct ServedMesh {
    vp_nf* nf = nullptr;          // resident near-field build
    bool owned = false;           // built by the server (cold registration)
    vp_mesh* mesh = nullptr;      // owned mesh of a cold registration
    std::vector<double> vxy;      // host copies of a cold registration
    std::vector<int32_t> tri;
    int32_t rule = VP_RULE_19_D9;
};

struct DevScope {
    int prev = -1;
    explicit DevScope(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevScope() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct vp_server {
    vp_ctx* ctx = nullptr;
    int precision = VP_MIXED;
    int64_t budget = 0;
    std::vector<cudaStream_t> streams;
    cudaStream_t build_stream = nullptr;       // cold-mesh builds
    std::vector<int64_t> slot_req;             // ticket running on each slot, -1 if free
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Req> reqs;
    std::unordered_map<int64_t, ServedMesh> meshes;
    int64_t next_ticket = 1;
    int64_t in_use = 0, peak_in_use = 0;
    int64_t completed = 0, failed = 0, evals_done = 0, cold_builds = 0;
    double t_first = -1, t_last_done = 0;
    std::vector<double> latency_ms, wait_ms;
    int max_running = 0;
    bool stop = false;
    std::thread worker;
    int magic = 0x56505356;
};

static int64_t footprint(const vp_ctx* ctx, const vp_nf* nf, int d, int precision) {
    const int64_t fb = (int64_t)d * nf->mesh->N * 8, ub = (int64_t)d * nf->M * 8;
    return ((fb + 255) & ~255LL) + ((ub + 255) & ~255LL) + (int64_t)eval_ws_bytes(ctx, nf, d, precision);
}

// Upload and build a cold mesh (called by the worker with the lock released).
static int build_cold(vp_server* sv, ServedMesh& m) {
    vp_mesh* mesh = nullptr;
    int rc = vp_mesh_upload(sv->ctx, m.vxy.data(), (int64_t)m.vxy.size() / 2, m.tri.data(), (int64_t)m.tri.size() / 3,
                            m.rule, (void*)sv->build_stream, &mesh);
    if (rc) return rc;
    vp_nf* nf = nullptr;
    rc = vp_nearfield_build(sv->ctx, mesh, 1, nullptr, 0, nullptr, (void*)sv->build_stream, &nf);
    if (rc) {
        vp_mesh_release(mesh);
        return rc;
    }
    if (sv->precision == VP_MIXED_FMM) {
        rc = fmm_plan_build(sv->ctx, nf, sv->build_stream);   // the multipole plan before the first request
        if (rc) {
            vp_nf_release(nf);
            vp_mesh_release(mesh);
            return rc;
        }
    }
    if (sv->precision == VP_MIXED && far_sym_applicable(nf, 1)) {
        rc = far_sym_plan(sv->ctx, nf);
        if (rc) {
            vp_nf_release(nf);
            vp_mesh_release(mesh);
            return rc;
        }
    }
    m.mesh = mesh;
    m.nf = nf;
    m.owned = true;
    return VP_OK;
}

static void worker_loop(vp_server* sv) {
    DevScope dg(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        bool progressed = false;
        // 1. completions
        for (size_t s = 0; s < sv->streams.size(); s++) {
            const int64_t t = sv->slot_req[s];
            if (t < 0) continue;
            Req& r = sv->reqs[t];
            const cudaError_t q = cudaEventQuery(r.ev);
            if (q == cudaErrorNotReady) continue;
            r.t_done = now_s();
            r.state = q == cudaSuccess ? RQ_DONE : RQ_FAILED;
            r.status = q == cudaSuccess ? VP_OK : VP_ERR_CUDA;
            cudaFreeAsync(r.dmem, sv->streams[s]);
            cudaEventDestroy(r.ev);
            r.dmem = nullptr;
            sv->in_use -= r.bytes;
            sv->slot_req[s] = -1;
            if (r.state == RQ_DONE) {
                sv->completed++;
                sv->evals_done += r.evals;
                sv->latency_ms.push_back(1e3 * (r.t_done - r.t_submit));
                sv->wait_ms.push_back(1e3 * (r.t_admit - r.t_submit));
            } else {
                sv->failed++;
            }
            sv->t_last_done = r.t_done;
            progressed = true;
        }
        if (progressed) sv->cv_done.notify_all();
        // 2. admissions, first come first served
        while (!sv->queue.empty()) {
            int slot = -1;
            for (size_t s = 0; s < sv->streams.size(); s++)
                if (sv->slot_req[s] < 0) {
                    slot = (int)s;
                    break;
                }
            if (slot < 0) break;
            const int64_t t = sv->queue.front();
            Req& r = sv->reqs[t];
            ServedMesh& m = sv->meshes[r.key];
            if (!m.nf) {
                // cold mesh: build it with the lock released (in-flight work continues)
                lk.unlock();
                const int rc = build_cold(sv, m);
                lk.lock();
                sv->cold_builds++;
                if (rc) {
                    sv->queue.pop_front();
                    r.state = RQ_FAILED;
                    r.status = rc;
                    r.t_done = now_s();
                    sv->failed++;
                    sv->cv_done.notify_all();
                    continue;
                }
            }
            const vp_nf* nf = m.nf;
            const int64_t need = footprint(sv->ctx, nf, r.d, sv->precision);
            if (need > sv->budget) {
                sv->queue.pop_front();
                r.state = RQ_FAILED;
                r.status = VP_ERR_OOM;
                r.t_done = now_s();
                sv->failed++;
                sv->cv_done.notify_all();
                continue;
            }
            if (sv->in_use + need > sv->budget) break;      // wait for memory to free up
            sv->queue.pop_front();
            cudaStream_t st = sv->streams[slot];
            void* mem = nullptr;
            if (cudaMallocAsync(&mem, (size_t)need, st) != cudaSuccess) {
                r.state = RQ_FAILED;
                r.status = VP_ERR_OOM;
                r.t_done = now_s();
                sv->failed++;
                sv->cv_done.notify_all();
                continue;
            }
            const int64_t fb = ((int64_t)r.d * nf->mesh->N * 8 + 255) & ~255LL;
            const int64_t ub = ((int64_t)r.d * nf->M * 8 + 255) & ~255LL;
            double* fd = (double*)mem;
            double* ud = (double*)((char*)mem + fb);
            void* ws = (char*)mem + fb + ub;
            cudaMemcpyAsync(fd, r.f_host, (size_t)r.d * nf->mesh->N * 8, cudaMemcpyHostToDevice, st);
            int rc = eval_impl(sv->ctx, nf, fd, r.d, ud, sv->precision, st, ws, false);
            cudaMemcpyAsync(r.u_host, ud, (size_t)r.d * nf->M * 8, cudaMemcpyDeviceToHost, st);
            cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
            cudaEventRecord(r.ev, st);
            r.dmem = mem;
            r.bytes = need;
            r.slot = slot;
            r.state = RQ_RUNNING;
            r.status = rc;
            r.t_admit = now_s();
            r.evals = (int64_t)r.d * nf->M;
            sv->in_use += need;
            sv->peak_in_use = std::max(sv->peak_in_use, sv->in_use);
            sv->slot_req[slot] = t;
            int running = 0;
            for (int64_t x : sv->slot_req) running += x >= 0;
            sv->max_running = std::max(sv->max_running, running);
            progressed = true;
        }
        bool busy = false;
        for (int64_t x : sv->slot_req) busy |= x >= 0;
        if (sv->stop && !busy && sv->queue.empty()) break;
        if (!progressed) {
            // poll running work every 50 us; sleep until a submission when idle
            if (busy || !sv->queue.empty()) sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else sv->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

extern "C" {

int vp_server_create(vp_ctx* ctx, int32_t slots, int64_t hbm_budget_bytes, int32_t precision, vp_server** out) {
    if (out) *out = nullptr;
    if (!ctx || ctx->magic != 0x56504358) return VP_ERR_STATE;
    if (!out || slots < 1 || slots > 64 || hbm_budget_bytes <= 0 ||
        (precision != VP_FP64 && precision != VP_MIXED && precision != VP_MIXED_FMM))
        return vp_set_error(ctx, VP_ERR_INVALID_ARG, "vp_server_create: bad arguments");
    DevScope dg(ctx->device);
    vp_server* sv = new (std::nothrow) vp_server();
    if (!sv) return VP_ERR_OOM;
    sv->ctx = ctx;
    sv->precision = precision;
    sv->budget = hbm_budget_bytes;
    for (int i = 0; i < slots; i++) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
            delete sv;
            return vp_set_error(ctx, VP_ERR_CUDA, "vp_server_create: stream creation failed");
        }
        sv->streams.push_back(s);
        sv->slot_req.push_back(-1);
    }
    if (cudaStreamCreateWithFlags(&sv->build_stream, cudaStreamNonBlocking) != cudaSuccess) {
        for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
        delete sv;
        return vp_set_error(ctx, VP_ERR_CUDA, "vp_server_create: stream creation failed");
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return VP_OK;
}

int vp_server_register(vp_server* sv, int64_t key, const vp_nf* nf) {
    if (!sv || sv->magic != 0x56505356) return VP_ERR_STATE;
    if (!nf || nf->magic != 0x56504e46 || nf->ctx != sv->ctx)
        return vp_set_error(sv->ctx, VP_ERR_STATE, "vp_server_register: bad near-field handle");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->meshes.count(key)) return vp_set_error(sv->ctx, VP_ERR_INVALID_ARG, "vp_server_register: key in use");
    if (sv->precision == VP_MIXED_FMM && !nf->fmm) {
        // the multipole plan is built here, before requests reach the mesh
        const int rc = fmm_plan_build(sv->ctx, const_cast<vp_nf*>(nf), sv->build_stream);
        if (rc) return rc;
    }
    if (sv->precision == VP_MIXED && far_sym_applicable(nf, 1) && !nf->sym) {
        // the symmetric far sum's unit tables, for its one-density requests
        const int rc = far_sym_plan(sv->ctx, const_cast<vp_nf*>(nf));
        if (rc) return rc;
    }
    ServedMesh m;
    m.nf = const_cast<vp_nf*>(nf);
    sv->meshes[key] = std::move(m);
    return VP_OK;
}

int vp_server_register_cold(vp_server* sv, int64_t key, const double* vxy, int64_t nv, const int32_t* tri, int64_t nt,
                            int32_t rule) {
    if (!sv || sv->magic != 0x56505356) return VP_ERR_STATE;
    if (!vxy || !tri || nv < 3 || nt < 1 || (rule != VP_RULE_16_D8 && rule != VP_RULE_19_D9))
        return vp_set_error(sv->ctx, VP_ERR_INVALID_ARG, "vp_server_register_cold: bad arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->meshes.count(key)) return vp_set_error(sv->ctx, VP_ERR_INVALID_ARG, "vp_server_register_cold: key in use");
    ServedMesh m;
    m.vxy.assign(vxy, vxy + 2 * nv);
    m.tri.assign(tri, tri + 3 * nt);
    m.rule = rule;
    sv->meshes[key] = std::move(m);
    return VP_OK;
}

int vp_server_mesh_size(vp_server* sv, int64_t key, int64_t* n_nodes, int64_t* n_targets) {
    if (!sv || sv->magic != 0x56505356) return VP_ERR_STATE;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->meshes.find(key);
    if (it == sv->meshes.end()) return vp_set_error(sv->ctx, VP_ERR_INVALID_ARG, "vp_server_mesh_size: unknown key");
    const ServedMesh& m = it->second;
    if (m.nf) {
        if (n_nodes) *n_nodes = m.nf->mesh->N;
        if (n_targets) *n_targets = m.nf->M;
    } else {
        const int64_t N = (int64_t)(m.tri.size() / 3) * m.rule;
        if (n_nodes) *n_nodes = N;
        if (n_targets) *n_targets = N;
    }
    return VP_OK;
}

int vp_server_submit(vp_server* sv, int64_t key, const double* f_host, int32_t d, double* u_host, int64_t* ticket) {
    if (ticket) *ticket = 0;
    if (!sv || sv->magic != 0x56505356) return VP_ERR_STATE;
    if (!f_host || !u_host || !ticket || d < 1 || d > 256)
        return vp_set_error(sv->ctx, VP_ERR_INVALID_ARG, "vp_server_submit: bad arguments");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (!sv->meshes.count(key)) return vp_set_error(sv->ctx, VP_ERR_INVALID_ARG, "vp_server_submit: unknown mesh key");
        const int64_t t = sv->next_ticket++;
        Req r;
        r.key = key;
        r.f_host = f_host;
        r.u_host = u_host;
        r.d = d;
        r.t_submit = now_s();
        if (sv->t_first < 0) sv->t_first = r.t_submit;
        sv->reqs[t] = r;
        sv->queue.push_back(t);
        *ticket = t;
    }
    sv->cv_work.notify_one();
    return VP_OK;
}

int vp_server_wait(vp_server* sv, int64_t ticket, double timeout_s, int32_t* status, double* latency_ms) {
    if (!sv || sv->magic != 0x56505356) return VP_ERR_STATE;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return vp_set_error(sv->ctx, VP_ERR_INVALID_ARG, "vp_server_wait: unknown ticket");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (it->second.state == RQ_QUEUED || it->second.state == RQ_RUNNING) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            (it->second.state == RQ_QUEUED || it->second.state == RQ_RUNNING))
            return VP_ERR_TIMEOUT;
    }
    if (status) *status = it->second.status;
    if (latency_ms) *latency_ms = 1e3 * (it->second.t_done - it->second.t_submit);
    return VP_OK;
}

static double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double fr = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - fr) + v[i + 1] * fr : v[i];
}

int vp_server_stats(vp_server* sv, vp_server_stats_t* out) {
    if (!sv || sv->magic != 0x56505356) return VP_ERR_STATE;
    if (!out) return VP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->queued = (int64_t)sv->queue.size();
    out->cold_builds = sv->cold_builds;
    out->evals = sv->evals_done;
    out->peak_bytes = sv->peak_in_use;
    out->max_concurrent = sv->max_running;
    out->p50_ms = percentile(sv->latency_ms, 0.50);
    out->p99_ms = percentile(sv->latency_ms, 0.99);
    out->p50_wait_ms = percentile(sv->wait_ms, 0.50);
    const double span = sv->t_first >= 0 ? sv->t_last_done - sv->t_first : 0.0;
    out->evals_per_s = span > 0 ? sv->evals_done / span : 0.0;
    return VP_OK;
}

void vp_server_destroy(vp_server* sv) {
    if (!sv || sv->magic != 0x56505356) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    DevScope dg(sv->ctx->device);
    for (cudaStream_t s : sv->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    cudaStreamSynchronize(sv->build_stream);
    cudaStreamDestroy(sv->build_stream);
    for (auto& kv : sv->meshes)
        if (kv.second.owned) {
            vp_nf_release(kv.second.nf);
            vp_mesh_release(kv.second.mesh);
        }
    sv->magic = 0;
    delete sv;
}

}  // extern "C"
