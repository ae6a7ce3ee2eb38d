// batch_api.cu -- the batched ensemble entry points of include/turret.h:
// many independent runs advanced by one launch per phase of the step.
//
// Each run keeps its own context (workspace, particle, window, storage).  A
// batch holds in device memory one RunDesc per run and, per phase, a prefix
// table of the blocks each run needs; block b of a batched launch serves run r
// with prefix[r] <= b < prefix[r + 1].  The step graph has the shape of the
// single-run graph with every node covering all runs:
//
//   batch stream: --fork--> bulk collide+stream (far cells: FP32 runs, then
//                           16-bit runs on x-pairs) --------------------------> join
//   side stream :       \-> near collide+stream -> particle + markers
//                           -> support moments + tile lists -> interpolation
//                           + rows of A -> cycles -> spread ---------------^
//   aux stream  :                         \-> F, T of every run (FP64) ---^
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <set>
#include <string>
#include <vector>

#include "../../include/turret.h"
#include "turret_ctx.cuh"
#include "turret_internal.cuh"

using namespace turret;

namespace {

enum { T_BULK = 0, T_NEAR, T_PM, T_MB, T_IP, T_CYC, T_SP, T_BULK16, T_COUNT };

std::string g_batch_init_err;

}  // namespace

struct turret_batch {
    int n;
    std::vector<turret_ctx *> ctx;
    cudaStream_t stream, side, aux;
    cudaEvent_t ev_fork, ev_join, ev_red, ev_red_done, ev_done, ev_pred;
    std::vector<cudaEvent_t> ev_ctx;  // one per run: the work already on its context's stream
    RunDesc *d_runs;
    CollideDesc *d_cdesc;             // the collide+stream part of each descriptor
    std::vector<CollideDesc> h_cdesc;
    int *d_prefix;                    // T_COUNT tables of n + 1 ints
    std::vector<RunDesc> h_runs;
    std::vector<int> h_prefix;
    int total[T_COUNT];
    int threads, minb, cycles, predictor, warm;
    long long step;
    cudaGraphExec_t graph[2];
    bool graph_ready[2];
    std::string err;
};

static turret_status bfail(turret_batch *b, turret_status s, const std::string &msg) {
    if (b) b->err = msg; else g_batch_init_err = msg;
    return s;
}

#define BK(call, where)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return bfail(b, TURRET_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CE(call)                          \
    do {                                  \
        cudaError_t e_ = (call);          \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

static size_t prefix_offset(int n) { return ((size_t)n * sizeof(RunDesc) + 255) & ~(size_t)255; }
static size_t cdesc_offset(int n) {
    return (prefix_offset(n) + (size_t)T_COUNT * (n + 1) * sizeof(int) + 255) & ~(size_t)255;
}

extern "C" size_t turret_batch_workspace_bytes(int32_t n) {
    if (n < 1) return 0;
    return cdesc_offset(n) + (size_t)n * sizeof(CollideDesc) + 256;
}

// Per-phase block tables from the descriptors and the launch shape.
static bool build_tables(turret_batch *b) {
    const int n = b->n;
    b->h_prefix.assign((size_t)T_COUNT * (n + 1), 0);
    for (int t = 0; t < T_COUNT; ++t) {
        long long acc = 0;
        for (int r = 0; r < n; ++r) {
            const RunDesc &R = b->h_runs[r];
            int k = 0;
            switch (t) {
                case T_BULK: k = blocks_bulk(R, b->threads); break;
                case T_NEAR: k = blocks_near(R, b->threads); break;
                case T_PM: k = blocks_particle_markers(R); break;
                case T_MB: k = blocks_box_moments_bin(R); break;
                case T_IP: k = blocks_interp0(R); break;
                case T_CYC: k = blocks_cycle(R); break;
                case T_SP: k = blocks_spread(R); break;
                default: k = blocks_bulk16(R); break;
            }
            b->h_prefix[(size_t)t * (n + 1) + r] = (int)acc;
            acc += k;
            if (acc >= (1LL << 31) - 1) return false;
        }
        b->h_prefix[(size_t)t * (n + 1) + n] = (int)acc;
        b->total[t] = (int)acc;
    }
    return true;
}

static void drop_batch_graphs(turret_batch *b) {
    for (int k = 0; k < 2; ++k) {
        if (b->graph_ready[k]) cudaGraphExecDestroy(b->graph[k]);
        b->graph_ready[k] = false;
    }
}

static cudaError_t upload(turret_batch *b) {
    b->h_cdesc.resize(b->n);
    for (int r = 0; r < b->n; ++r) {
        const RunDesc &R = b->h_runs[r];
        CollideDesc &D = b->h_cdesc[r];
        memset(&D, 0, sizeof D);
        D.g = R.g;
        D.box = R.box;
        for (int k = 0; k < 2; ++k) {
            D.f[k] = R.f[k];
            D.utop[k] = R.utop[k];
        }
        D.st = R.st;
        D.hbox = R.ba.h;
        D.storage = R.storage;
        D.split = R.split;
        D.tx = R.tx;
        D.tx16 = bulk16_tile(R);
    }
    CE(cudaMemcpyAsync(b->d_runs, b->h_runs.data(), b->n * sizeof(RunDesc), cudaMemcpyHostToDevice, b->stream));
    CE(cudaMemcpyAsync(b->d_cdesc, b->h_cdesc.data(), b->n * sizeof(CollideDesc), cudaMemcpyHostToDevice,
                       b->stream));
    CE(cudaMemcpyAsync(b->d_prefix, b->h_prefix.data(), b->h_prefix.size() * sizeof(int), cudaMemcpyHostToDevice,
                       b->stream));
    return cudaStreamSynchronize(b->stream);
}

static void release_batch(turret_batch *b) {
    if (!b) return;
    drop_batch_graphs(b);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->aux) cudaStreamDestroy(b->aux);
    cudaEvent_t evs[6] = {b->ev_fork, b->ev_join, b->ev_red, b->ev_red_done, b->ev_done, b->ev_pred};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_ctx)
        if (e) cudaEventDestroy(e);
    delete b;
}

extern "C" turret_status turret_batch_init(turret_batch **out, turret_ctx *const *ctxs, int32_t n, void *ws,
                                           size_t ws_bytes, void *stream) {
    turret_batch *b = nullptr;
    if (!out) return bfail(b, TURRET_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return bfail(b, TURRET_EINVAL, "no runs");
    std::set<const turret_ctx *> seen;
    for (int r = 0; r < n; ++r) {
        const turret_ctx *c = ctxs[r];
        if (!c) return bfail(b, TURRET_EINVAL, "NULL context in the run list");
        if (!seen.insert(c).second) return bfail(b, TURRET_EINVAL, "a context appears twice");
        if (!c->has_particle) return bfail(b, TURRET_ESTATE, "every run needs a loaded surface");
        if ((c->step & 1) != (ctxs[0]->step & 1)) return bfail(b, TURRET_ESTATE, "runs at time levels of different parity");
        if (c->flags.ibm_cycles != ctxs[0]->flags.ibm_cycles)
            return bfail(b, TURRET_EINVAL, "runs with different ibm_cycles");
        if ((c->body.predictor != 0) != (ctxs[0]->body.predictor != 0))
            return bfail(b, TURRET_EINVAL, "runs with and without a force predictor");
        if (c->body.predictor != 0 && ((c->body.pred_opts ^ ctxs[0]->body.pred_opts) & PRED_WARM))
            return bfail(b, TURRET_EINVAL, "runs with and without warm-started IBM cycles");
    }
    if (!ws || ws_bytes < turret_batch_workspace_bytes(n)) return bfail(b, TURRET_ENOMEM, "batch workspace too small");
    if (((uintptr_t)ws & 255) != 0) return bfail(b, TURRET_EINVAL, "workspace must be 256-byte aligned");

    b = new turret_batch();
    b->n = n;
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = (cudaStream_t)stream;
    b->side = b->aux = nullptr;
    b->ev_fork = b->ev_join = b->ev_red = b->ev_red_done = b->ev_done = b->ev_pred = nullptr;
    b->graph_ready[0] = b->graph_ready[1] = false;
    b->d_runs = (RunDesc *)ws;
    b->d_prefix = (int *)((char *)ws + prefix_offset(n));
    b->d_cdesc = (CollideDesc *)((char *)ws + cdesc_offset(n));
    b->threads = 128;
    b->minb = 2;
    b->cycles = ctxs[0]->flags.ibm_cycles;
    b->predictor = ctxs[0]->body.predictor != 0 ? 1 : 0;
    b->warm = (b->predictor && (ctxs[0]->body.pred_opts & PRED_WARM)) ? 1 : 0;
    b->step = ctxs[0]->step;
    b->h_runs.resize(n);
    for (int r = 0; r < n; ++r) {
        const turret_ctx *c = ctxs[r];
        RunDesc &R = b->h_runs[r];
        memset(&R, 0, sizeof R);
        R.g = c->geom;
        R.bc = c->body;
        R.box = c->box;
        R.m = c->mk;
        R.ba = c->ba;
        for (int k = 0; k < 2; ++k) {
            R.f[k] = c->f[k];
            R.utop[k] = c->utop[k];
        }
        R.st = c->dstate;
        R.tile_list = c->tile_list;
        R.tile_count = c->tile_count;
        R.storage = c->storage;
        R.cap = c->cap;
        R.nm = c->nm;
        R.split = c->split ? 1 : 0;
        R.tx = 32;
        const MlpDev *net = mlp_device_view(c->net);
        if (c->body.predictor == 2 && net) R.mlp = *net;
    }
    if (!build_tables(b)) {
        release_batch(b);
        return bfail(nullptr, TURRET_EINVAL, "too many blocks in one batched launch");
    }
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->aux, cudaStreamNonBlocking, hi);
    cudaEvent_t *evs[6] = {&b->ev_fork, &b->ev_join, &b->ev_red, &b->ev_red_done, &b->ev_done, &b->ev_pred};
    for (cudaEvent_t *ev : evs)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    b->ev_ctx.assign(n, nullptr);
    for (int r = 0; r < n && e == cudaSuccess; ++r) e = cudaEventCreateWithFlags(&b->ev_ctx[r], cudaEventDisableTiming);
    // the contexts' pending work (e.g. their initial coupling) precedes the upload
    for (int r = 0; r < n && e == cudaSuccess; ++r) {
        e = cudaEventRecord(b->ev_ctx[r], ctxs[r]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_ctx[r], 0);
    }
    if (e == cudaSuccess) e = upload(b);
    if (e != cudaSuccess) {
        release_batch(b);
        return bfail(nullptr, TURRET_ECUDA, std::string("turret_batch_init: ") + cudaGetErrorString(e));
    }
    *out = b;
    return TURRET_OK;
}

extern "C" turret_status turret_batch_set_tiles(turret_batch *b, int32_t threads, int32_t minb, const int32_t *tx) {
    if (!b) return bfail(b, TURRET_EINVAL, "NULL batch");
    if (!tx) return bfail(b, TURRET_EINVAL, "NULL tile list");
    for (int r = 0; r < b->n; ++r)
        if (!valid_tile(threads, tx[r], minb)) return bfail(b, TURRET_EINVAL, "invalid launch shape");
    const int old_threads = b->threads;
    std::vector<int> old_tx(b->n);
    for (int r = 0; r < b->n; ++r) {
        old_tx[r] = b->h_runs[r].tx;
        b->h_runs[r].tx = tx[r];
    }
    b->threads = threads;
    if (!build_tables(b)) {
        b->threads = old_threads;
        for (int r = 0; r < b->n; ++r) b->h_runs[r].tx = old_tx[r];
        build_tables(b);
        return bfail(b, TURRET_EINVAL, "too many blocks in one batched launch");
    }
    b->minb = minb;
    drop_batch_graphs(b);
    BK(upload(b), "set_tiles upload");
    return TURRET_OK;
}

// One batched step from parity p (every run: f[p] holds f*(t-1)).
static cudaError_t batch_enqueue(turret_batch *b, int p) {
    const int n = b->n;
    auto tab = [&](int t) { return (const int *)(b->d_prefix + (size_t)t * (n + 1)); };
    const RunDesc *R = b->d_runs;
    CE(cudaEventRecord(b->ev_fork, b->stream));
    CE(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    // the predictions and the particle/marker updates run on the aux stream
    // beside the near collide+stream
    CE(cudaStreamWaitEvent(b->aux, b->ev_fork, 0));
    if (b->predictor) CE(launch_batch_predict(R, n, p, b->aux));
    CE(launch_batch_particle_markers(R, tab(T_PM), n, p, b->total[T_PM], b->aux));
    CE(cudaEventRecord(b->ev_pred, b->aux));
    CE(launch_batch_collide(PHASE_BULK, b->d_cdesc, tab(T_BULK), n, p, b->total[T_BULK], b->threads, b->minb,
                            b->stream));
    CE(launch_batch_collide(PHASE_BULK16, b->d_cdesc, tab(T_BULK16), n, p, b->total[T_BULK16], 128, 5, b->stream));
    CE(launch_batch_collide(PHASE_NEAR, b->d_cdesc, tab(T_NEAR), n, p, b->total[T_NEAR], b->threads, 1, b->side));
    CE(cudaStreamWaitEvent(b->side, b->ev_pred, 0));
    CE(launch_batch_box_moments_bin(R, tab(T_MB), n, p, b->total[T_MB], b->side));
    CE(launch_batch_interp0(R, tab(T_IP), n, b->total[T_IP], b->warm, b->side));
    CE(cudaEventRecord(b->ev_red, b->side));
    CE(cudaStreamWaitEvent(b->aux, b->ev_red, 0));
    CE(launch_batch_reduce_ft(R, n, p ^ 1, b->aux));
    CE(cudaEventRecord(b->ev_red_done, b->aux));
    if (!b->warm) {
        // the paper's cycles: h^0 = r0, then 1 .. n-1 alternating so that the last writes hl
        const int C = b->cycles - 1;
        int src = HSEL_R0;
        for (int cyc = 1; cyc <= C; ++cyc) {
            const int dst = ((C - cyc) % 2 == 0) ? HSEL_HL : HSEL_HB;
            CE(launch_batch_cycle(R, tab(T_CYC), n, b->total[T_CYC], src, dst, -1, cyc == C, cyc - 1, 0, b->side));
            src = dst;
        }
    } else {
        // predictor modes: up to n adaptive cycles from the previous h
        const int C = b->cycles;
        int src = HSEL_HL;
        for (int cyc = 1; cyc <= C; ++cyc) {
            const int dst = (cyc % 2 == 1) ? HSEL_HB : HSEL_HL;
            const int fin = (cyc == C && dst != HSEL_HL) ? HSEL_HL : -1;
            CE(launch_batch_cycle(R, tab(T_CYC), n, b->total[T_CYC], src, dst, fin, cyc == C, cyc - 1, 1, b->side));
            src = dst;
        }
    }
    CE(launch_batch_spread(R, tab(T_SP), n, b->total[T_SP], b->side));
    CE(cudaStreamWaitEvent(b->side, b->ev_red_done, 0));
    CE(cudaEventRecord(b->ev_join, b->side));
    CE(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
    return cudaSuccess;
}

// The bulk collide+stream node low, every other kernel node (the chain) high.
static void set_batch_priorities(cudaGraph_t gr) {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return;
    size_t cnt = 0;
    if (cudaGraphGetNodes(gr, nullptr, &cnt) != cudaSuccess || cnt == 0) return;
    std::vector<cudaGraphNode_t> nodes(cnt);
    if (cudaGraphGetNodes(gr, nodes.data(), &cnt) != cudaSuccess) return;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        cudaLaunchAttributeValue v;
        memset(&v, 0, sizeof v);
        v.priority = is_batch_bulk_kernel(kp.func) ? lo : hi;
        cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v);
    }
    cudaGetLastError();  // priorities are a hint; never fail a step on them
}

extern "C" turret_status turret_batch_step(turret_batch *b, int64_t nsteps) {
    if (!b) return bfail(b, TURRET_EINVAL, "NULL batch");
    if (nsteps < 0) return bfail(b, TURRET_EINVAL, "negative step count");
    if (nsteps == 0) return TURRET_OK;
    // runs may also be stepped alone between batched steps (all state is on
    // the device) as long as their time levels keep one parity
    for (int r = 0; r < b->n; ++r)
        if ((b->ctx[r]->step & 1) != (b->ctx[0]->step & 1))
            return bfail(b, TURRET_ESTATE, "runs at time levels of different parity");
    b->step = b->ctx[0]->step;
    for (int r = 0; r < b->n; ++r) {
        BK(cudaEventRecord(b->ev_ctx[r], b->ctx[r]->stream), "order after run streams");
        BK(cudaStreamWaitEvent(b->stream, b->ev_ctx[r], 0), "order after run streams");
    }
    const bool graphs = b->stream != nullptr;
    for (int64_t k = 0; k < nsteps; ++k) {
        const int p = (int)(b->step & 1);
        if (graphs) {
            if (!b->graph_ready[p]) {
                cudaGraph_t gr;
                BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                cudaError_t e = batch_enqueue(b, p);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
                if (e != cudaSuccess) {
                    if (e2 == cudaSuccess) cudaGraphDestroy(gr);
                    return bfail(b, TURRET_ECUDA, std::string("capture enqueue: ") + cudaGetErrorString(e));
                }
                BK(e2, "end capture");
                set_batch_priorities(gr);
                e = cudaGraphInstantiateWithFlags(&b->graph[p], gr, cudaGraphInstantiateFlagUseNodePriority);
                cudaGraphDestroy(gr);
                BK(e, "graph instantiate");
                b->graph_ready[p] = true;
            }
            BK(cudaGraphLaunch(b->graph[p], b->stream), "graph launch");
        } else {
            BK(batch_enqueue(b, p), "batched step launch");
        }
        b->step++;
    }
    for (int r = 0; r < b->n; ++r) b->ctx[r]->step += nsteps;
    BK(cudaEventRecord(b->ev_done, b->stream), "order run streams after the batch");
    for (int r = 0; r < b->n; ++r)
        BK(cudaStreamWaitEvent(b->ctx[r]->stream, b->ev_done, 0), "order run streams after the batch");
    return TURRET_OK;
}

extern "C" turret_status turret_batch_destroy(turret_batch *b) {
    if (!b) return TURRET_EINVAL;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->side) cudaStreamSynchronize(b->side);
    if (b->aux) cudaStreamSynchronize(b->aux);
    release_batch(b);
    return TURRET_OK;
}

extern "C" const char *turret_batch_last_error(const turret_batch *b) {
    return b ? b->err.c_str() : g_batch_init_err.c_str();
}

// ---------------------------------------------------------------------------
// Tile timing for the autotuner.  From time level t (parity p) the kernel
// reads f[p] and the ghost velocity utop[1 - p] and writes f[1 - p] and
// utop[p]: both hold values no later call reads before the next step
// overwrites them, so the timed launches leave the context's state unchanged.
extern "C" turret_status turret_time_collide(turret_ctx *c, int32_t threads, int32_t tx, int32_t minb, int32_t reps,
                                             float *us_out) {
    if (!c || !us_out) return TURRET_EINVAL;
    if (!valid_tile(threads, tx, minb) || reps < 1 || reps > 100000) {
        c->err = "invalid launch shape or repetition count";
        return TURRET_EINVAL;
    }
    const int p = (int)(c->step & 1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto launch = [&]() {
        return launch_collide_tiled(c->geom, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate,
                                    p, c->has_particle ? c->ba.h : nullptr, c->box, c->has_particle, threads, tx, minb,
                                    c->stream);
    };
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        c->err = std::string("turret_time_collide: ") + cudaGetErrorString(e);
        return TURRET_ECUDA;
    }
    *us_out = 1000.0f * ms / (float)reps;
    return TURRET_OK;
}
