// turret_api.cu -- the extern "C" boundary of libturret.so (include/turret.h):
// context creation over caller-owned device workspaces, surface loading with
// host FP64 mesh properties, and the per-step launch sequence captured as one
// CUDA graph per ping-pong parity.
//
// Step graph (time t -> t+1, parity p = t % 2), when the particle's near
// region fits the window:
//
//   caller stream: --fork--> collide+stream, far cells ------------------> join
//   side stream  :       \-> collide+stream, near cells -+-> support moments
//                           + tile lists -> interpolation + rows of A
//                           -> (h <- h + r0 - A h) x (n-1) -> spread h_imm(t+1) --^
//   aux stream   :       \-> [prediction] -> particle update + markers -/
//                                                    ... -> F, T (FP64) ----^
//
// The near region (support box grown by two cells) contains every cell the
// next support-box pull reads, so the immersed-boundary chain only waits for
// the small near launch and runs concurrently with the bulk of the window
// (the side stream has the highest priority).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <stdio.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/turret.h"
#include "turret_ctx.cuh"
#include "turret_internal.cuh"

using namespace turret;

static std::string g_init_err;

static turret_status fail(turret_ctx *c, turret_status s, const std::string &msg) {
    if (c) c->err = msg; else g_init_err = msg;
    return s;
}

static turret_status cuda_fail(turret_ctx *c, cudaError_t e, const char *where) {
    cudaGetLastError();  // a non-sticky error must not surface in later launches
    return fail(c, TURRET_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where);  \
    } while (0)

#define CE(call)                                \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

// Sequential 256-byte-aligned carving of a caller workspace (or size count).
struct Carver {
    char *base;
    size_t off;
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

static bool valid_window(const turret_window *w) {
    if (!w || w->nx < 1 || w->ny < 1 || w->nz < 1) return false;
    if (w->bc_x < 0 || w->bc_x > 1 || w->bc_y < 0 || w->bc_y > 1) return false;
    if (w->bc_bottom < 0 || w->bc_bottom > 3 || w->bc_bottom == TURRET_BC_PRESSURE || w->bc_top < 0 ||
        w->bc_top > 3)
        return false;
    if (w->slide && (w->bc_bottom == TURRET_BC_MOVING || w->bc_top == TURRET_BC_MOVING)) return false;
    if ((w->bc_bottom == TURRET_BC_PERIODIC) != (w->bc_top == TURRET_BC_PERIODIC)) return false;
    if (w->sponge_cells < 0 || w->sponge_cells > w->nz) return false;
    if (w->slide && (w->bc_bottom == TURRET_BC_PERIODIC)) return false;
    if (w->slide && !(w->anchor_frac > 0.0 && w->anchor_frac < 1.0)) return false;
    if (w->nz > 65535) return false;
    if ((long long)w->nx * w->ny * w->nz > (1LL << 31) / 27) return false;
    return true;
}

static void carve_fluid(Carver &cv, const turret_window *w, int st, void **f, float **utop, DevState **ds,
                        float **tau_z) {
    const size_t ncell = (size_t)w->nx * w->ny * w->nz, plane = (size_t)w->nx * w->ny;
    for (int k = 0; k < 2; ++k) f[k] = cv.take(27 * ncell * storage_bytes(st));
    for (int k = 0; k < 2; ++k) utop[k] = (float *)cv.take(3 * plane * sizeof(float));
    *ds = (DevState *)cv.take(sizeof(DevState));
    *tau_z = (float *)cv.take(2 * (size_t)w->nz * sizeof(float));  // tau, then 1/tau, per plane
}

extern "C" size_t lbm_workspace_bytes(const turret_window *win, turret_storage st) {
    if (!valid_window(win) || st < 0 || st > 2) return 0;
    Carver cv{nullptr, 0};
    void *f[2];
    float *u[2];
    DevState *ds;
    float *tz;
    carve_fluid(cv, win, (int)st, f, u, &ds, &tz);
    return cv.off + 256;
}

static void release(turret_ctx *c) {
    if (!c) return;
    for (int k = 0; k < 2; ++k) {
        if (c->graph_ready[k]) cudaGraphExecDestroy(c->graph[k]);
        if (c->multi_ready[k]) cudaGraphExecDestroy(c->graph_multi[k]);
    }
    if (c->side) cudaStreamDestroy(c->side);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_red) cudaEventDestroy(c->ev_red);
    if (c->ev_red_done) cudaEventDestroy(c->ev_red_done);
    if (c->ev_pred) cudaEventDestroy(c->ev_pred);
    cudaEvent_t *xs[6] = {c->ev_far, c->ev_near, c->ev_pm, c->ev_ired, c->ev_redd, c->ev_spread};
    for (cudaEvent_t *x : xs)
        for (int k = 0; k < 2; ++k)
            if (x[k]) cudaEventDestroy(x[k]);
    if (c->pinned) cudaFreeHost(c->pinned);
    delete c;
}

extern "C" turret_status lbm_init(turret_ctx **out, const turret_window *win, turret_lattice lat, double nu,
                                  double rho_ratio, const double g[3], turret_storage st, void *ws,
                                  size_t ws_bytes, void *stream) {
    turret_ctx *c = nullptr;
    if (!out) return fail(c, TURRET_EINVAL, "out is NULL");
    *out = nullptr;
    if (lat != TURRET_D3Q27) return fail(c, TURRET_EINVAL, "only the D3Q27 lattice is supported");
    if (!valid_window(win)) return fail(c, TURRET_EINVAL, "invalid window");
    if (st < 0 || st > 2) return fail(c, TURRET_EINVAL, "invalid storage");
    const double tau = 3.0 * nu + 0.5;  // nu = c_s^2 (tau - 1/2), Eq. 9
    if (!(nu > 0.0) || !(tau > 0.5) || !isfinite(tau)) return fail(c, TURRET_EINVAL, "nu must give tau > 1/2");
    if (!(rho_ratio > 0.0) || !isfinite(rho_ratio)) return fail(c, TURRET_EINVAL, "rho_ratio must be positive");
    if (!g || !isfinite(g[0]) || !isfinite(g[1]) || !isfinite(g[2])) return fail(c, TURRET_EINVAL, "invalid g");
    const size_t need = lbm_workspace_bytes(win, st);
    if (!ws || ws_bytes < need) return fail(c, TURRET_ENOMEM, "fluid workspace too small");
    if (((uintptr_t)ws & 255) != 0) return fail(c, TURRET_EINVAL, "workspace must be 256-byte aligned");

    c = new turret_ctx();
    c->side = c->aux = nullptr;
    c->ev_fork = c->ev_join = c->ev_red = c->ev_red_done = c->ev_pred = nullptr;
    for (int k = 0; k < 2; ++k) {
        c->ev_far[k] = c->ev_near[k] = c->ev_pm[k] = c->ev_ired[k] = c->ev_redd[k] = c->ev_spread[k] = nullptr;
        c->multi_ready[k] = false;
    }
    c->pred_mode = 0;
    c->pred_opts = 0;
    c->pred_eps = 0.0f;
    c->pred_theta = INFINITY;
    c->net = nullptr;
    c->log = nullptr;
    c->log_cap = 0;
    c->pinned = nullptr;
    c->graph_ready[0] = c->graph_ready[1] = false;
    c->win = *win;
    memset(&c->flags, 0, sizeof c->flags);
    c->flags.ibm_cycles = 4;
    c->reinject = Reinject{0, 0, 0, 0};
    c->storage = (int)st;
    c->nu = nu;
    c->tau0 = tau;
    c->kappa = rho_ratio;
    for (int a = 0; a < 3; ++a) c->g[a] = g[a];
    c->stream = (cudaStream_t)stream;
    Geom &G = c->geom;
    G.nx = win->nx; G.ny = win->ny; G.nz = win->nz;
    G.bc_x = win->bc_x; G.bc_y = win->bc_y; G.bc_bottom = win->bc_bottom; G.bc_top = win->bc_top;
    G.sponge = win->sponge_cells;
    G.plane = (long long)win->nx * win->ny;
    G.ncell = G.plane * win->nz;
    G.tau0 = (float)tau;
    G.force_scheme = 0;
    G.sround = 0;
    for (int a = 0; a < 3; ++a) G.uw_bottom[a] = G.uw_top[a] = 0.0f;
    Carver cv{(char *)ws, 0};
    float *tau_z = nullptr;
    carve_fluid(cv, win, c->storage, c->f, c->utop, &c->dstate, &tau_z);
    // relaxation time per logical plane: tau0, rising linearly to 1 on the top
    // plane over the sponge (Sec. 2.5), tabulated in double and stored as float
    c->tau_host.assign(2 * (size_t)win->nz, 0.0f);
    for (int z = 0; z < win->nz; ++z) {
        double t = tau;
        const int L = win->sponge_cells;
        if (L > 0 && z >= win->nz - L) t = tau + (1.0 - tau) * (double)(z - (win->nz - L) + 1) / (double)L;
        c->tau_host[z] = (float)t;
        c->tau_host[win->nz + z] = (float)(1.0 / t);
    }
    G.tau_z = tau_z;
    G.omega_z = tau_z + win->nz;
    // 16-bit storage on a window the staged collide+stream tiles: tensor maps
    // of both population buffers (plain loads if the driver refuses them)
    c->staged = staged_eligible(G, c->storage) && prepare_staged();
    for (int k = 0; k < 2 && c->staged; ++k)
        c->staged = encode_population_map(&c->lmap[k], c->f[k], G, true) &&
                    encode_population_map(&c->smap[k], c->f[k], G, false);
    c->has_particle = false;
    c->split = false;
    c->step = 0;
    if (cudaMallocHost((void **)&c->pinned, sizeof(DevState)) != cudaSuccess) {
        c->pinned = nullptr;  // queries then stage through pageable memory
        cudaGetLastError();
    }
    int lo_prio = 0, hi_prio = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, hi_prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_red, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_red_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_pred, cudaEventDisableTiming);
    {
        cudaEvent_t *xs[6] = {c->ev_far, c->ev_near, c->ev_pm, c->ev_ired, c->ev_redd, c->ev_spread};
        for (cudaEvent_t *x : xs)
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&x[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tau_z, c->tau_host.data(), c->tau_host.size() * sizeof(float), cudaMemcpyHostToDevice,
                            c->stream);
    // fluid at rest: all deviations zero, ghost velocity zero, window state reset
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(c->f[k], 0, 27 * (size_t)G.ncell * storage_bytes(c->storage), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->utop[k], 0, 3 * (size_t)G.plane * sizeof(float), c->stream);
    }
    memset(&c->host_state, 0, sizeof(DevState));
    for (int k = 0; k < 2; ++k) {
        for (int i = 0; i < 9; ++i) c->host_state.s[k].d[i] = (i % 4 == 0) ? 1.0 : 0.0;
        c->host_state.s[k].reseed = -1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->dstate, &c->host_state, sizeof(DevState), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "lbm_init");
        release(c);
        return TURRET_ECUDA;
    }
    *out = c;
    return TURRET_OK;
}

static void drop_graphs(turret_ctx *c) {
    for (int k = 0; k < 2; ++k) {
        if (c->graph_ready[k]) cudaGraphExecDestroy(c->graph[k]);
        if (c->multi_ready[k]) cudaGraphExecDestroy(c->graph_multi[k]);
        c->graph_ready[k] = false;
        c->multi_ready[k] = false;
    }
}

extern "C" turret_status lbm_set_flags(turret_ctx *c, const turret_flags *fl) {
    if (!c || !fl) return fail(c, TURRET_EINVAL, "NULL argument");
    if (fl->force_scheme < 0 || fl->force_scheme > 1 || fl->rot_form < 0 || fl->rot_form > 1 || fl->gravity < 0 ||
        fl->gravity > 1 || fl->ibm_cycles < 1 || fl->ibm_cycles > 64 || fl->stochastic_rounding < 0 ||
        fl->stochastic_rounding > 1 || fl->fixed_position < 0 || fl->fixed_position > 1 || fl->force_eval < 0 ||
        fl->force_eval > 1)
        return fail(c, TURRET_EINVAL, "invalid flags");
    if (c->has_particle) return fail(c, TURRET_ESTATE, "flags must be set before ibm_load_surface");
    c->flags = *fl;
    c->geom.force_scheme = fl->force_scheme;
    c->geom.sround = (c->storage == ST_BF16 && fl->stochastic_rounding) ? 1 : 0;
    drop_graphs(c);
    return TURRET_OK;
}

extern "C" turret_status lbm_set_wall_velocity(turret_ctx *c, const double u_bottom[3], const double u_top[3]) {
    if (!c || !u_bottom || !u_top) return fail(c, TURRET_EINVAL, "NULL argument");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(u_bottom[a]) || !isfinite(u_top[a]) || fabs(u_bottom[a]) > 0.3 || fabs(u_top[a]) > 0.3)
            return fail(c, TURRET_EINVAL, "wall speed must be finite and below 0.3");
    if (u_bottom[2] != 0.0 || u_top[2] != 0.0) return fail(c, TURRET_EINVAL, "walls move in their plane only");
    for (int a = 0; a < 3; ++a) {
        c->geom.uw_bottom[a] = (float)u_bottom[a];
        c->geom.uw_top[a] = (float)u_top[a];
    }
    drop_graphs(c);
    return TURRET_OK;
}

extern "C" turret_status lbm_set_fields(turret_ctx *c, const double *rho, const double *u) {
    if (!c) return fail(c, TURRET_EINVAL, "NULL context");
    if (c->has_particle) return fail(c, TURRET_ESTATE, "fields must be set before ibm_load_surface");
    const size_t n = (size_t)c->geom.ncell;
    const int p = (int)(c->step & 1);
    double *dr = (double *)c->f[1 - p];  // the idle buffer holds >= 54 bytes per cell
    double *du = dr + n;
    std::vector<double> h(n);
    if (rho) {
        for (size_t k = 0; k < n; ++k) h[k] = rho[k] - 1.0;
        CK(cudaMemcpyAsync(dr, h.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "set_fields rho");
    }
    if (u) CK(cudaMemcpyAsync(du, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "set_fields u");
    CK(launch_init_equilibrium(c->geom, c->storage, c->f[p], rho ? dr : nullptr, u ? du : nullptr,
                               c->utop[1 - p], c->stream),
       "init_equilibrium");
    CK(cudaStreamSynchronize(c->stream), "set_fields sync");
    return TURRET_OK;
}

// ---------------------------------------------------------------------------
// Host FP64 surface properties: dS_k (one third of the adjacent triangle
// areas, Sec. 2.2), outward vertex normals (area-weighted), volume, centre of
// mass and J/m about it from the divergence theorem (every triangle closes a
// tetrahedron with the origin).
struct MeshProps {
    std::vector<double> dS, nrm;
    double vol, area, com[3], Jm[9];
};

static bool mesh_props(const double *V, int64_t nv, const int32_t *T, int64_t nt, MeshProps &mp) {
    std::map<std::pair<int64_t, int64_t>, int> edges;
    for (int64_t t = 0; t < nt; ++t)
        for (int e = 0; e < 3; ++e) {
            const int64_t a = T[3 * t + e], b = T[3 * t + (e + 1) % 3];
            if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) return false;
            if (++edges[{a, b}] > 1) return false;
        }
    for (auto &kv : edges)
        if (!edges.count({kv.first.second, kv.first.first})) return false;
    std::vector<int> used(nv, 0);
    for (int64_t t = 0; t < 3 * nt; ++t) used[T[t]] = 1;
    for (int64_t k = 0; k < nv; ++k)
        if (!used[k]) return false;
    mp.dS.assign(nv, 0.0);
    mp.nrm.assign(3 * nv, 0.0);
    double vol = 0.0, area = 0.0, s1[3] = {0, 0, 0}, s2[9] = {0};
    for (int64_t t = 0; t < nt; ++t) {
        const double *p0 = V + 3 * T[3 * t], *p1 = V + 3 * T[3 * t + 1], *p2 = V + 3 * T[3 * t + 2];
        const double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        const double w[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        const double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double ar = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        area += ar;
        for (int e = 0; e < 3; ++e) {
            const int64_t k = T[3 * t + e];
            mp.dS[k] += ar / 3.0;
            for (int a = 0; a < 3; ++a) mp.nrm[3 * k + a] += 0.5 * cr[a];
        }
        // signed volume of the tetrahedron (0, p0, p1, p2) = p0 . (p1 x p2) / 6
        const double c12[3] = {p1[1] * p2[2] - p1[2] * p2[1], p1[2] * p2[0] - p1[0] * p2[2],
                               p1[0] * p2[1] - p1[1] * p2[0]};
        const double tv = (p0[0] * c12[0] + p0[1] * c12[1] + p0[2] * c12[2]) / 6.0;
        vol += tv;
        double sum[3];
        for (int a = 0; a < 3; ++a) {
            sum[a] = p0[a] + p1[a] + p2[a];
            s1[a] += tv * sum[a] * 0.25;
        }
        // second moments of a tetrahedron with one vertex at the origin
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                s2[3 * a + b] += tv * 0.05 * (p0[a] * p0[b] + p1[a] * p1[b] + p2[a] * p2[b] + sum[a] * sum[b]);
    }
    if (!(vol > 0.0)) return false;
    for (int64_t k = 0; k < nv; ++k) {
        double *n = &mp.nrm[3 * k];
        const double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(l > 0.0)) return false;
        for (int a = 0; a < 3; ++a) n[a] /= l;
    }
    for (int a = 0; a < 3; ++a) mp.com[a] = s1[a] / vol;
    double C[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[3 * a + b] = s2[3 * a + b] - vol * mp.com[a] * mp.com[b];
    const double tr = C[0] + C[4] + C[8];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) mp.Jm[3 * a + b] = ((a == b) ? tr : 0.0) / vol - C[3 * a + b] / vol;
    mp.vol = vol;
    mp.area = area;
    return true;
}

static bool inverse3(const double *A, double *B) {
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(fabs(det) > 0.0)) return false;
    const double id = 1.0 / det;
    B[0] = (A[4] * A[8] - A[5] * A[7]) * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = (A[5] * A[6] - A[3] * A[8]) * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = (A[3] * A[7] - A[4] * A[6]) * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return true;
}

struct IbmLayout {
    BoxGeom box;
    int nm, cap, rc;
    double rmin, rmax;
};

// Support box: every marker lies within rc = ceil(bounding radius) of C_m,
// so all 4x4x4 stencils fit a cube of 2 rc + 6 cells placed at floor(C) - rc - 2;
// rc includes the offset F_OFFSET of the stress surface (its stencils too).
static bool ibm_layout(const MeshProps &mp, const double *V, int64_t nv, IbmLayout &L) {
    if (nv <= 0 || nv >= (1 << 24)) return false;
    double rb = 0.0, rs = INFINITY;
    for (int64_t k = 0; k < nv; ++k) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (V[3 * k + a] - mp.com[a]) * (V[3 * k + a] - mp.com[a]);
        rb = fmax(rb, sqrt(s));
        rs = fmin(rs, sqrt(s));
    }
    L.rmin = rs;
    L.rmax = rb;
    // 1e-3: margin for the FP32 rounding of the marker positions on the GPU
    // (their stencils must stay off the box's outer layer)
    L.rc = (int)ceil(rb + F_OFFSET + 1e-3);
    const int B = 2 * L.rc + 6;
    L.box.Bx = L.box.By = L.box.Bz = B;
    L.box.tx = L.box.ty = L.box.tz = (B + TILE - 1) / TILE;
    L.box.nbox = (long long)B * B * B;
    L.nm = (int)nv;
    L.cap = (int)(nv < MAX_CANDIDATES ? nv : MAX_CANDIDATES);
    return B <= 1024;
}

static size_t carve_ibm(Carver &cv, const IbmLayout &L, turret_ctx *c) {
    const size_t nm = (size_t)L.nm, nb = (size_t)L.box.nbox;
    const size_t ntiles = (size_t)L.box.tx * L.box.ty * L.box.tz;
    MarkerArrays m;
    m.Xb = (const float *)cv.take(3 * nm * 4);
    m.nb = (const float *)cv.take(3 * nm * 4);
    m.dS = (const float *)cv.take(nm * 4);
    m.dSo = (const float *)cv.take(nm * 4);
    m.rec = (MRec *)cv.take(nm * sizeof(MRec));
    m.reco = (MRec *)cv.take(nm * sizeof(MRec));
    m.base = (int *)cv.take(nm * 4);
    m.ft = (float *)cv.take(9 * nm * 4);
    m.U = (float *)cv.take(3 * nm * 4);
    m.n = (float *)cv.take(3 * nm * 4);
    m.arm = (float *)cv.take(3 * nm * 4);
    m.hl = (float *)cv.take(3 * nm * 4);
    m.r0 = (float *)cv.take(3 * nm * 4);
    m.hb = (float *)cv.take(3 * nm * 4);
    m.aval = (float *)cv.take(nm * (size_t)ROWCAP * 4);
    m.aidx = (int *)cv.take(nm * (size_t)ROWCAP * 4);
    m.alen = (int *)cv.take(nm * 4);
    m.seg = (int *)cv.take(6 * ((nm + MARKER_SEG - 1) / MARKER_SEG) * 4);
    m.force_eval = c ? c->flags.force_eval : 0;
    BoxArrays ba;
    ba.u = (float *)cv.take(3 * nb * 4);
    ba.s = (float *)cv.take(6 * nb * 4);
    ba.p = (float *)cv.take(nb * 4);
    ba.h = (float *)cv.take(3 * nb * 4);
    int *tl = (int *)cv.take(2 * ntiles * (size_t)L.cap * 4);  // spreading list, rows-of-A list
    int *tc = (int *)cv.take(2 * ntiles * 4);
    if (c) {
        c->mk = m;
        c->ba = ba;
        c->tile_list = tl;
        c->tile_count = tc;
    }
    return cv.off + 256;
}

extern "C" size_t ibm_workspace_bytes(const turret_ctx *c, const double *V, int64_t nv, const int32_t *T,
                                      int64_t nt) {
    if (!c || !V || !T || nv <= 0 || nt <= 0) return 0;
    MeshProps mp;
    if (!mesh_props(V, nv, T, nt, mp)) return 0;
    IbmLayout L;
    if (!ibm_layout(mp, V, nv, L)) return 0;
    Carver cv{nullptr, 0};
    return carve_ibm(cv, L, nullptr);
}

// Events (2)-(4) of Table 1.  advance = 1: particle update t -> t+1 from
// window slot `slot` (markers land in slot^1), then u* and sigma on the
// support box from f(t+1) = pull(f*(t)) together with the tile candidate
// lists, the surface force and torque, and n IBM cycles -> h_imm(t+1).
// advance = 0: the same at the current time level (slot `slot`) without
// moving the particle (set-up of t = 0).
// The IBM cycles of one step (the paper's n - 1 cycles from r0, or the
// warm-started adaptive ones) on stream s.
static cudaError_t enqueue_cycles(turret_ctx *c, int warm, cudaStream_t s) {
    const int nm = c->nm;
    if (!warm) {
        // the paper's cycles: h^0 = r0, then cycles 1 .. n-1 alternating so
        // that the last one writes hl
        const int C = c->flags.ibm_cycles - 1;
        const float *src = c->mk.r0;
        for (int cyc = 1; cyc <= C; ++cyc) {
            float *dst = ((C - cyc) % 2 == 0) ? c->mk.hl : c->mk.hb;
            CE(launch_cycle(nm, c->mk, src, dst, nullptr, cyc == C, c->dstate, cyc - 1, 0, 0.0f, s));
            src = dst;
        }
    } else {
        // predictor modes: up to n cycles from the previous h (in hl), each
        // skipped once the slip is below the tolerance; hl ends with the result
        const int C = c->flags.ibm_cycles;
        const float *src = c->mk.hl;
        for (int cyc = 1; cyc <= C; ++cyc) {
            float *dst = (cyc % 2 == 1) ? c->mk.hb : c->mk.hl;
            float *fin = (cyc == C && dst != c->mk.hl) ? c->mk.hl : nullptr;
            CE(launch_cycle(nm, c->mk, src, dst, fin, cyc == C, c->dstate, cyc - 1, 1, c->body.slip_eps, s));
            src = dst;
        }
    }
    return cudaSuccess;
}

// pm_done: when non-null, the particle/marker update was already enqueued
// (on the aux stream, beside the near collide+stream) and this event marks it.
static cudaError_t enqueue_coupling(turret_ctx *c, const void *fsrc, const float *utop_in, int slot, int advance,
                                    cudaStream_t s, cudaEvent_t pm_done = nullptr) {
    const int nm = c->nm;
    const int so = advance ? (slot ^ 1) : slot;
    const bool branch = (s == c->side);  // reduce F, T on the aux branch
    if (pm_done) CE(cudaStreamWaitEvent(s, pm_done, 0));
    else CE(launch_particle_markers(c->geom, c->body, c->box, c->dstate, slot, advance, c->mk, s));
    CE(launch_box_moments_bin(c->geom, c->storage, fsrc, utop_in, c->dstate, so, c->box, c->ba, nm, c->mk.base, c->mk.seg,
                              c->tile_list, c->tile_count, c->cap, c->dstate, c->body.rmin, c->body.rmax, s));
    const int warm = (advance && c->body.predictor != 0 && (c->body.pred_opts & PRED_WARM)) ? 1 : 0;
    CE(launch_interp0(c->box, nm, c->mk, c->ba, c->tile_list, c->tile_count, c->cap, c->dstate, warm, s));
    if (branch) {
        CE(cudaEventRecord(c->ev_red, s));
        CE(cudaStreamWaitEvent(c->aux, c->ev_red, 0));
        CE(launch_reduce_ft(nm, c->mk, c->dstate, so, c->body, c->aux));
        CE(cudaEventRecord(c->ev_red_done, c->aux));
    } else {
        CE(launch_reduce_ft(nm, c->mk, c->dstate, so, c->body, s));
    }
    CE(enqueue_cycles(c, warm, s));
    CE(launch_spread(c->box, nm, c->mk, c->ba, c->tile_list, c->tile_count, c->cap, s));
    if (branch) CE(cudaStreamWaitEvent(s, c->ev_red_done, 0));
    return cudaSuccess;
}

// Tensor maps of the staged 16-bit collide+stream from f[p] into f[1 - p]
// (source boxes of f[p], destination boxes of f[1 - p]) when the window can be
// staged and flags.staged_loads asks for it, else null (plain loads and stores).
static const CUtensorMap *src_map(const turret_ctx *c, int p) {
    return (c->staged && c->flags.staged_loads) ? &c->lmap[p] : nullptr;
}
static const CUtensorMap *dst_map(const turret_ctx *c, int p) {
    return (c->staged && c->flags.staged_loads) ? &c->smap[1 - p] : nullptr;
}

// Collide+stream over the whole window without forcing (no particle), the
// window slot carried to slot_out.
static cudaError_t collide_window(const turret_ctx *c, int p, cudaStream_t s) {
    if (src_map(c, p))
        return launch_collide_staged(c->geom, c->storage, *src_map(c, p), *dst_map(c, p), c->f[p], c->f[1 - p],
                                     c->utop[1 - p], c->utop[p], c->dstate, p, 1 - p, nullptr, c->box, REGION_ALL,
                                     s);
    if (xpair_eligible(c->geom, c->storage))
        return launch_collide_xpair(c->geom, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate,
                                    p, 1 - p, nullptr, c->box, REGION_ALL, s);
    return launch_collide_stream(c->geom, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate, p,
                                 1 - p, nullptr, c->box, false, REGION_ALL, s);
}

// One step from parity p: f[p] holds f*(t-1), f[1-p] receives f*(t).
static cudaError_t enqueue_step(turret_ctx *c, int p) {
    const Geom &G = c->geom;
    if (!c->has_particle) return collide_window(c, p, c->stream);
    if (c->reinject.trigger > 0) {
        // re-injection copy: collide+stream over the whole window, the particle
        // and marker update, the copy of f*(t) (the buffer of f*(t-1) stages
        // it) with the window shift, then the chain
        if (c->body.predictor != 0)
            CE(launch_predict(c->body.predictor == 2 ? mlp_device_view(c->net) : nullptr, c->dstate, p,
                              c->body.predictor, c->stream));
        CE(launch_collide_stream(G, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate, p, -1,
                                 c->ba.h, c->box, true, REGION_ALL, c->stream));
        CE(launch_particle_markers(G, c->body, c->box, c->dstate, p, 1, c->mk, c->stream));
        CE(launch_reinject(G, c->storage, c->f[1 - p], c->f[p], c->dstate, 1 - p, c->reinject, c->stream));
        CE(cudaEventRecord(c->ev_pred, c->stream));
        return enqueue_coupling(c, c->f[1 - p], c->utop[p], p, 1, c->stream, c->ev_pred);
    }
    cudaStream_t chain = c->split ? c->side : c->stream;
    const bool predict = c->body.predictor != 0;
    const MlpDev *net = (c->body.predictor == 2) ? mlp_device_view(c->net) : nullptr;
    if (c->split) {
        // the prediction and the particle/marker update (which reads only the
        // body state) run on the aux stream beside the near collide+stream
        CE(cudaEventRecord(c->ev_fork, c->stream));
        CE(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        CE(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
        if (predict) CE(launch_predict(net, c->dstate, p, c->body.predictor, c->aux));
        CE(launch_particle_markers(c->geom, c->body, c->box, c->dstate, p, 1, c->mk, c->aux));
        CE(cudaEventRecord(c->ev_pred, c->aux));
        CE(launch_collide_far(G, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate, p, c->ba.h,
                              c->box, c->stream, src_map(c, p), dst_map(c, p)));
        CE(launch_collide_stream(G, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate, p, -1,
                                 c->ba.h, c->box, true, REGION_NEAR, c->side));
    } else {
        if (predict) CE(launch_predict(net, c->dstate, p, c->body.predictor, c->stream));
        CE(launch_collide_stream(G, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate, p, -1,
                                 c->ba.h, c->box, true, REGION_ALL, c->stream));
    }
    CE(enqueue_coupling(c, c->f[1 - p], c->utop[p], p, 1, chain, c->split ? c->ev_pred : nullptr));
    if (c->split) {
        CE(cudaEventRecord(c->ev_join, c->side));
        CE(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    }
    return cudaSuccess;
}

// Steps t .. t+K-1 (parity p0 first) as one capture with the exact cross-step
// dependencies (split windows only), so the immersed-boundary chain of step
// t overlaps the far-cell collide+stream of step t+1:
//   far(t)    after near(t-1) [its near-region cells of f*(t-1)] and pm(t-1)
//             [the window slot of t];
//   pm(t)     (prediction + particle/marker update, aux) after far(t-1) and
//             near(t-1) [they read the slot pm(t) writes] and spread(t-1)
//             [the marker arrays pm(t) rewrites], and reduce(t-1) [F, T];
//   near(t)   after far(t-1) [its far-cell sources and the buffer it writes];
//   moments(t) after near(t) and pm(t); the chain then as in one step;
//   reduce(t) (aux) after interpolation(t).
// Each event is recorded once per step parity; a wait always refers to the
// step the dependency names.  Per-step results equal those of one-step graphs.
static cudaError_t enqueue_steps_pipelined(turret_ctx *c, int p0, int K) {
    const Geom &G = c->geom;
    const int nm = c->nm;
    const bool predict = c->body.predictor != 0;
    const MlpDev *net = (c->body.predictor == 2) ? mlp_device_view(c->net) : nullptr;
    CE(cudaEventRecord(c->ev_fork, c->stream));
    CE(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    CE(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    int p = p0;
    for (int k = 0; k < K; ++k, p ^= 1) {
        const int q = p ^ 1;
        const bool first = k == 0;
        // caller stream: the far cells of step t
        if (!first) {
            CE(cudaStreamWaitEvent(c->stream, c->ev_near[q], 0));
            CE(cudaStreamWaitEvent(c->stream, c->ev_pm[q], 0));
        }
        CE(launch_collide_far(G, c->storage, c->f[p], c->f[q], c->utop[q], c->utop[p], c->dstate, p, c->ba.h, c->box,
                              c->stream, src_map(c, p), dst_map(c, p)));
        CE(cudaEventRecord(c->ev_far[p], c->stream));
        // aux: prediction and particle/marker update
        if (!first) {
            CE(cudaStreamWaitEvent(c->aux, c->ev_far[q], 0));
            CE(cudaStreamWaitEvent(c->aux, c->ev_spread[q], 0));
        }
        if (predict) CE(launch_predict(net, c->dstate, p, c->body.predictor, c->aux));
        CE(launch_particle_markers(G, c->body, c->box, c->dstate, p, 1, c->mk, c->aux));
        CE(cudaEventRecord(c->ev_pm[p], c->aux));
        // side: the near cells, then the immersed-boundary chain
        if (!first) CE(cudaStreamWaitEvent(c->side, c->ev_far[q], 0));
        CE(launch_collide_stream(G, c->storage, c->f[p], c->f[q], c->utop[q], c->utop[p], c->dstate, p, -1, c->ba.h,
                                 c->box, true, REGION_NEAR, c->side));
        CE(cudaEventRecord(c->ev_near[p], c->side));
        CE(cudaStreamWaitEvent(c->side, c->ev_pm[p], 0));
        CE(launch_box_moments_bin(G, c->storage, c->f[q], c->utop[p], c->dstate, q, c->box, c->ba, nm, c->mk.base,
                                  c->mk.seg, c->tile_list, c->tile_count, c->cap, c->dstate, c->body.rmin,
                                  c->body.rmax, c->side));
        const int warm = (c->body.predictor != 0 && (c->body.pred_opts & PRED_WARM)) ? 1 : 0;
        CE(launch_interp0(c->box, nm, c->mk, c->ba, c->tile_list, c->tile_count, c->cap, c->dstate, warm, c->side));
        CE(cudaEventRecord(c->ev_ired[p], c->side));
        CE(cudaStreamWaitEvent(c->aux, c->ev_ired[p], 0));
        CE(launch_reduce_ft(nm, c->mk, c->dstate, q, c->body, c->aux));
        CE(cudaEventRecord(c->ev_redd[p], c->aux));
        CE(enqueue_cycles(c, warm, c->side));
        CE(launch_spread(c->box, nm, c->mk, c->ba, c->tile_list, c->tile_count, c->cap, c->side));
        CE(cudaEventRecord(c->ev_spread[p], c->side));
    }
    const int last = p ^ 1;
    CE(cudaStreamWaitEvent(c->stream, c->ev_spread[last], 0));
    CE(cudaStreamWaitEvent(c->stream, c->ev_redd[last], 0));
    return cudaSuccess;
}

extern "C" turret_status ibm_load_surface(turret_ctx *c, const double *V, int64_t nv, const int32_t *T, int64_t nt,
                                          const double r0[3], const double v0[3], const double w0[3], void *ws,
                                          size_t ws_bytes) {
    if (!c) return fail(c, TURRET_EINVAL, "NULL context");
    if (c->has_particle) return fail(c, TURRET_ESTATE, "a surface is already loaded");
    if (!V || !T || nv <= 0 || nt <= 0 || !r0 || !v0 || !w0) return fail(c, TURRET_EINVAL, "invalid surface arguments");
    MeshProps mp;
    if (!mesh_props(V, nv, T, nt, mp))
        return fail(c, TURRET_EINVAL, "surface is not a closed, outward-oriented triangle mesh");
    IbmLayout L;
    if (!ibm_layout(mp, V, nv, L)) return fail(c, TURRET_EINVAL, "too many markers or too large a surface");
    const int n[3] = {c->win.nx, c->win.ny, c->win.nz};
    const bool per[3] = {c->win.bc_x == 0, c->win.bc_y == 0, c->win.bc_bottom == 0};
    bool split = true;
    for (int a = 0; a < 3; ++a) {
        if (per[a] && L.box.Bx > n[a])
            return fail(c, TURRET_EINVAL, "support box wider than the window along a periodic axis");
        if (per[a] && L.box.Bx + 2 * NEAR_GROW > n[a]) split = false;
    }
    // every marker stencil must start inside the window along closed axes
    for (int64_t k = 0; k < nv; ++k)
        for (int a = 0; a < 3; ++a) {
            if (per[a]) continue;
            const double X = r0[a] + (V[3 * k + a] - mp.com[a]);
            const int b = (int)floor(X);
            if (b - 1 < 0 || b + 2 > n[a] - 1)
                return fail(c, TURRET_EINVAL, "a marker is closer than 2 cells to a closed face");
            const int bo = (int)floor(X + (c->flags.force_eval == 0 ? F_OFFSET * mp.nrm[3 * k + a] : 0.0));
            if (bo - 1 < 0 || bo + 2 > n[a] - 1)
                return fail(c, TURRET_EINVAL, "a point of the stress surface is closer than 2 cells to a closed face");
        }
    double Jinv[9];
    if (!inverse3(mp.Jm, Jinv)) return fail(c, TURRET_EINVAL, "singular inertia tensor");
    Carver cv{(char *)ws, 0};
    const size_t need = carve_ibm(cv, L, nullptr);
    if (!ws || ws_bytes < need) return fail(c, TURRET_ENOMEM, "ibm workspace too small");
    if (((uintptr_t)ws & 255) != 0) return fail(c, TURRET_EINVAL, "workspace must be 256-byte aligned");
    Carver cv2{(char *)ws, 0};
    carve_ibm(cv2, L, c);
    c->nm = L.nm;
    c->cap = L.cap;
    c->box = L.box;
    c->vol = mp.vol;
    c->area = mp.area;
    c->split = split;
    BodyConst &B = c->body;
    B.vol = mp.vol;
    B.kappa = c->kappa;
    B.mass = c->kappa * mp.vol;
    B.inv_mass = 1.0 / B.mass;
    for (int i = 0; i < 9; ++i) B.Jinv_b[i] = Jinv[i] * B.inv_mass;
    for (int a = 0; a < 3; ++a) B.g_eff[a] = (c->flags.gravity == 1 ? 1.0 : 1.0 - 1.0 / c->kappa) * c->g[a];
    B.anchor_z = c->win.anchor_frac * c->win.nz;
    B.rot_form = c->flags.rot_form;
    B.fixed = c->flags.fixed_position;
    B.force_eval = c->flags.force_eval;
    B.renorm = c->flags.renorm_orientation;
    B.slide = c->win.slide;
    B.nm = L.nm;
    B.rc = L.rc;
    B.rmin = (float)L.rmin;
    B.rmax = (float)L.rmax;
    B.predictor = c->pred_mode;
    B.pred_opts = c->pred_opts;
    B.slip_eps = c->pred_eps;
    B.resid_theta = c->pred_theta;
    B.log = c->log;
    B.log_cap = c->log_cap;
    // static marker data (body frame): offsets from C_m, normals, areas
    const size_t nm = (size_t)L.nm;
    c->staging.assign(8 * nm, 0.0f);
    for (size_t k = 0; k < nm; ++k) {
        for (int a = 0; a < 3; ++a) {
            c->staging[a * nm + k] = (float)(V[3 * k + a] - mp.com[a]);
            c->staging[(3 + a) * nm + k] = (float)mp.nrm[3 * k + a];
        }
        c->staging[6 * nm + k] = (float)mp.dS[k];
    }
    // areas of the offset surface Xb + F_OFFSET nb: the same triangles, one
    // third of each triangle's area to each of its vertices
    for (int64_t t = 0; t < nt; ++t) {
        double P[3][3];
        for (int e = 0; e < 3; ++e)
            for (int a = 0; a < 3; ++a) P[e][a] = V[3 * T[3 * t + e] + a] + F_OFFSET * mp.nrm[3 * T[3 * t + e] + a];
        const double u[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
        const double w[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
        const double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double ar = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        for (int e = 0; e < 3; ++e) c->staging[7 * nm + T[3 * t + e]] += (float)(ar / 3.0);
    }
    CK(cudaMemcpyAsync((void *)c->mk.Xb, c->staging.data(), 3 * nm * 4, cudaMemcpyHostToDevice, c->stream), "Xb");
    CK(cudaMemcpyAsync((void *)c->mk.nb, c->staging.data() + 3 * nm, 3 * nm * 4, cudaMemcpyHostToDevice, c->stream),
       "nb");
    CK(cudaMemcpyAsync((void *)c->mk.dS, c->staging.data() + 6 * nm, nm * 4, cudaMemcpyHostToDevice, c->stream), "dS");
    CK(cudaMemcpyAsync((void *)c->mk.dSo, c->staging.data() + 7 * nm, nm * 4, cudaMemcpyHostToDevice, c->stream),
       "dSo");
    CK(cudaMemsetAsync(c->ba.h, 0, 3 * (size_t)L.box.nbox * 4, c->stream), "h");
    // the moments kernel skips the box cells no stencil reads: they keep
    // finite values (zeros, or an earlier step's moments)
    CK(cudaMemsetAsync(c->ba.u, 0, 3 * (size_t)L.box.nbox * 4, c->stream), "u");
    CK(cudaMemsetAsync(c->ba.s, 0, 6 * (size_t)L.box.nbox * 4, c->stream), "sigma");
    CK(cudaMemsetAsync(c->ba.p, 0, (size_t)L.box.nbox * 4, c->stream), "p");
    // rigid-body state at t: r(t), d = I, v(t-1/2) = v0, w(t-1/2) = w0, L = J w0
    CK(cudaMemcpyAsync(&c->host_state, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "state");
    CK(cudaStreamSynchronize(c->stream), "load sync");
    DevState &D = c->host_state;
    const int t = (int)(c->step & 1);
    BodySlot &S = D.s[t];
    for (int a = 0; a < 3; ++a) {
        S.r[a] = r0[a] + (double)S.origin[a];
        S.v[a] = v0[a];
        S.w[a] = w0[a];
        D.F[a] = D.T[a] = 0.0;
        S.L[a] = B.mass * (mp.Jm[3 * a] * w0[0] + mp.Jm[3 * a + 1] * w0[1] + mp.Jm[3 * a + 2] * w0[2]);
        const double C = r0[a];
        S.Ci[a] = (int)floor(C);
        S.Cf[a] = C - floor(C);
        S.box_lo[a] = S.Ci[a] - L.rc - 2;
        int lw = S.box_lo[a];
        if (per[a]) {
            lw %= n[a];
            if (lw < 0) lw += n[a];
        }
        S.box_lo_w[a] = lw;
    }
    for (int i = 0; i < 9; ++i) S.d[i] = (i % 4 == 0) ? 1.0 : 0.0;
    S.step = c->step;
    D.status = 0;
    D.counter = 0;
    CK(cudaMemcpyAsync(c->dstate, &D, sizeof(DevState), cudaMemcpyHostToDevice, c->stream), "state upload");
    c->has_particle = true;
    drop_graphs(c);
    CK(enqueue_coupling(c, c->f[t], c->utop[1 - t], t, 0, c->stream), "initial coupling");
    CK(cudaStreamSynchronize(c->stream), "initial coupling sync");
    return TURRET_OK;
}

// Stream priorities are not part of a captured graph: mark the bulk
// collide+stream node low and every other kernel node (the immersed-boundary
// chain on the critical path) high, so the chain's blocks are dispatched
// first whenever an SM frees up.
static void set_node_priorities(const turret_ctx *c, cudaGraph_t gr) {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return;
    size_t n = 0;
    if (cudaGraphGetNodes(gr, nullptr, &n) != cudaSuccess || n == 0) return;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(gr, nodes.data(), &n) != cudaSuccess) return;
    const dim3 bulk((c->geom.nx + 31) / 32, (c->geom.ny + 3) / 4, (c->geom.nz + 1) / 2);  // plane pairs
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        const bool is_bulk = (kp.gridDim.x == bulk.x && kp.gridDim.y == bulk.y && kp.gridDim.z == bulk.z &&
                              kp.blockDim.x == 32 && kp.blockDim.y == 4) ||
                             is_staged_kernel(kp.func) || is_xpair_kernel(kp.func);
        cudaLaunchAttributeValue v;
        memset(&v, 0, sizeof v);
        v.priority = is_bulk ? lo : hi;
        cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v);
    }
    cudaGetLastError();  // priorities are a hint; never fail a step on them
}

// Steps per replay of the pipelined multi-step graph (even: the parity after
// a replay is the one before it).
constexpr int PIPE_STEPS = 8;

static cudaError_t capture(turret_ctx *c, int p, int K, cudaGraphExec_t *out) {
    cudaGraph_t gr;
    CE(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = (K == 1) ? enqueue_step(c, p) : enqueue_steps_pipelined(c, p, K);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
    if (e != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(gr);
        return e;
    }
    CE(e2);
    set_node_priorities(c, gr);
    e = cudaGraphInstantiateWithFlags(out, gr, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(gr);
    return e;
}

extern "C" turret_status step(turret_ctx *c, int64_t n) {
    if (!c) return fail(c, TURRET_EINVAL, "NULL context");
    if (n < 0) return fail(c, TURRET_EINVAL, "negative step count");
    const bool graphs = (c->stream != nullptr) && !c->flags.no_graph;
    int64_t k = 0;
    if (graphs && c->has_particle && c->split && c->reinject.trigger == 0) {
        // whole groups of PIPE_STEPS steps as one pipelined graph
        for (; n - k >= PIPE_STEPS; k += PIPE_STEPS) {
            const int p = (int)(c->step & 1);
            if (!c->multi_ready[p]) {
                CK(capture(c, p, PIPE_STEPS, &c->graph_multi[p]), "multi-step capture");
                c->multi_ready[p] = true;
            }
            CK(cudaGraphLaunch(c->graph_multi[p], c->stream), "graph launch");
            c->step += PIPE_STEPS;
        }
    }
    for (; k < n; ++k) {
        const int p = (int)(c->step & 1);
        if (graphs) {
            if (!c->graph_ready[p]) {
                CK(capture(c, p, 1, &c->graph[p]), "capture");
                c->graph_ready[p] = true;
            }
            CK(cudaGraphLaunch(c->graph[p], c->stream), "graph launch");
        } else {
            CK(enqueue_step(c, p), "step launch");
        }
        c->step++;
    }
    return TURRET_OK;
}

extern "C" turret_status turret_set_predictor(turret_ctx *c, int32_t mode, const turret_mlp *net, int32_t options,
                                              double slip_eps, double resid_theta) {
    if (!c) return fail(c, TURRET_EINVAL, "NULL context");
    if (mode < 0 || mode > 2) return fail(c, TURRET_EINVAL, "predictor mode must be 0, 1 or 2");
    if (options < 0 || options > (PRED_WARM | PRED_VEL | PRED_REL))
        return fail(c, TURRET_EINVAL, "invalid predictor options");
    if (mode == 2 && !net) return fail(c, TURRET_EINVAL, "the network predictor needs a network");
    if (!(slip_eps >= 0.0) || !(resid_theta > 0.0)) return fail(c, TURRET_EINVAL, "invalid tolerances");
    c->pred_mode = mode;
    c->pred_opts = options;
    c->body.pred_opts = options;
    c->net = net;
    c->pred_eps = (float)slip_eps;
    c->pred_theta = resid_theta;
    c->body.predictor = mode;
    c->body.slip_eps = c->pred_eps;
    c->body.resid_theta = resid_theta;
    drop_graphs(c);
    return TURRET_OK;
}

extern "C" turret_status turret_set_reinjection(turret_ctx *c, int32_t trigger, int32_t target, int32_t below,
                                                int32_t above) {
    if (!c) return fail(c, TURRET_EINVAL, "NULL context");
    if (trigger != 0) {
        if (c->win.slide || c->win.bc_bottom == TURRET_BC_PERIODIC)
            return fail(c, TURRET_EINVAL, "re-injection needs a window without slide and a closed bottom");
        if (!(trigger > 0 && trigger < target && target < c->win.nz) || below < 0 || above < 0 ||
            below + above > c->win.nz)
            return fail(c, TURRET_EINVAL, "need 0 < trigger < target < nz and a block inside the window");
    }
    c->reinject = Reinject{trigger, target, below, above};
    drop_graphs(c);
    return TURRET_OK;
}

extern "C" turret_status turret_set_log(turret_ctx *c, double *records, int64_t capacity) {
    if (!c) return fail(c, TURRET_EINVAL, "NULL context");
    if (capacity < 0 || (capacity > 0 && !records)) return fail(c, TURRET_EINVAL, "invalid log");
    c->log = capacity > 0 ? records : nullptr;
    c->log_cap = capacity;
    c->body.log = c->log;
    c->body.log_cap = capacity;
    drop_graphs(c);
    return TURRET_OK;
}

extern "C" turret_status turret_query_predictor(turret_ctx *c, turret_predictor_stats *out) {
    if (!c || !out) return fail(c, TURRET_EINVAL, "NULL argument");
    DevState D;
    CK(cudaMemcpyAsync(&D, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "query");
    CK(cudaStreamSynchronize(c->stream), "query sync");
    memset(out, 0, sizeof *out);
    out->steps = D.pr.steps;
    out->net_steps = D.pr.mlp_steps;
    out->fallbacks = D.pr.fallbacks;
    out->cycles = D.pr.cycles;
    out->logged = D.pr.logged;
    out->resid = D.pr.resid;
    for (int k = 0; k < 8; ++k) {
        unsigned int b = D.pr.slip[k];
        float f;
        memcpy(&f, &b, 4);
        out->slip[k] = f;
    }
    out->hist_n = D.pr.hist_n;
    out->fallback = D.pr.fallback;
    return TURRET_OK;
}

extern "C" turret_status lbm_fluid_step(turret_ctx *c, int64_t n) {
    if (!c) return fail(c, TURRET_EINVAL, "NULL context");
    if (n < 0) return fail(c, TURRET_EINVAL, "negative step count");
    // the kernels of the coupled step's collide+stream as the step runs them:
    // the far cells on the context stream and the near region (which also
    // carries the body slot) beside them on the side stream, so that timing
    // this call times the step's own collide+stream
    const bool split = c->has_particle && c->split && c->reinject.trigger == 0;
    for (int64_t k = 0; k < n; ++k) {
        const int p = (int)(c->step & 1);
        if (split) {
            CK(cudaEventRecord(c->ev_fork, c->stream), "fluid step (fork)");
            CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fluid step (fork)");
            CK(launch_collide_far(c->geom, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate, p,
                                  c->ba.h, c->box, c->stream, src_map(c, p), dst_map(c, p)),
               "fluid step (far cells)");
            CK(launch_collide_stream(c->geom, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate,
                                     p, 1 - p, c->ba.h, c->box, true, REGION_NEAR, c->side),
               "fluid step (near region)");
            CK(cudaEventRecord(c->ev_join, c->side), "fluid step (join)");
            CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "fluid step (join)");
        } else if (!c->has_particle) {
            CK(collide_window(c, p, c->stream), "fluid step");
        } else {
            CK(launch_collide_stream(c->geom, c->storage, c->f[p], c->f[1 - p], c->utop[1 - p], c->utop[p], c->dstate,
                                     p, 1 - p, c->ba.h, c->box, true, REGION_ALL, c->stream),
               "fluid step");
        }
        c->step++;
    }
    return TURRET_OK;
}

extern "C" turret_status query_particle_state(turret_ctx *c, turret_particle_state *out) {
    if (!c || !out) return fail(c, TURRET_EINVAL, "NULL argument");
    DevState D;
    DevState *dst = c->pinned ? c->pinned : &D;
    CK(cudaMemcpyAsync(dst, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "query");
    CK(cudaStreamSynchronize(c->stream), "query sync");
    if (c->pinned) D = *c->pinned;
    const BodySlot &S = D.s[c->step & 1];  // the body at the current time level
    memset(out, 0, sizeof *out);
    for (int a = 0; a < 3; ++a) {
        out->r[a] = S.r[a];
        out->v[a] = S.v[a];
        out->w[a] = S.w[a];
        out->F[a] = D.F[a];
        out->T[a] = D.T[a];
        out->Fp[a] = D.Fp[a];
        out->L[a] = S.L[a];
        out->origin[a] = S.origin[a];
    }
    for (int i = 0; i < 9; ++i) out->d[i] = S.d[i];
    out->step = c->has_particle ? S.step : c->step;
    out->status = D.status;
    out->n_markers = c->has_particle ? c->nm : 0;
    out->volume = c->has_particle ? c->vol : 0.0;
    out->area = c->has_particle ? c->area : 0.0;
    // collide+stream (1, or far + near), particle + markers, moments + tile
    // lists, interpolation + rows of A, F/T reduction, one product per extra
    // cycle, spread of h_imm
    out->kernels_per_step = c->has_particle ? (c->split ? 2 : 1) + 5 + (c->flags.ibm_cycles - 1) +
                                                  (c->pred_mode != 0 ? 1 : 0) +  // prediction
                                                  ((c->pred_mode != 0 && (c->pred_opts & PRED_WARM)) ? 1 : 0)
                                            : 1;
    if (D.status == STAT_DOMAIN) return fail(c, TURRET_EDOMAIN, "a marker stencil left the window");
    if (D.status == STAT_DIVERGED) return fail(c, TURRET_EDIVERGED, "non-finite force or torque");
    if (D.status == STAT_OVERFLOW) return fail(c, TURRET_EOVERFLOW, "a support tile overflowed its marker list");
    if (D.status == STAT_TIMEOUT) return fail(c, TURRET_ETIMEOUT, "a staged copy did not complete in time");
    return TURRET_OK;
}

static turret_status copy_fields(turret_ctx *c, float *dev_out, bool pops) {
    if (!c || !dev_out) return fail(c, TURRET_EINVAL, "NULL argument");
    const int p = (int)(c->step & 1);
    CK(launch_macro(c->geom, c->storage, c->f[p], c->utop[1 - p], c->dstate, p, dev_out, pops, c->stream), "macro");
    CK(cudaStreamSynchronize(c->stream), "macro sync");
    return TURRET_OK;
}

extern "C" turret_status lbm_copy_macro(turret_ctx *c, float *dev_out) { return copy_fields(c, dev_out, false); }
extern "C" turret_status lbm_copy_populations(turret_ctx *c, float *dev_out) { return copy_fields(c, dev_out, true); }

// ---------------------------------------------------------------------------
// Checkpoints.  The state of a context at time level t (parity p = t % 2):
// the post-collision populations f*(t-1) in f[p] (storage precision as is),
// the top-plane ghost velocity in utop[1 - p], the device state (body and
// window slots, F, T, status, predictor history), h_imm(t) on the support
// box and the Lagrangian force h (hl, the warm start of the next cycles).
// Everything else a step reads is rebuilt by the step itself.
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, storage, has_particle, nm;
    turret_window win;
    turret_flags flags;
    double nu, kappa, g[3];
    int64_t step, nbox;
    int64_t bytes_pop, bytes_utop, bytes_state, bytes_h, bytes_hl;
};
const char CKPT_MAGIC[8] = {'T', 'U', 'R', 'R', 'E', 'T', 'C', 'K'};

// Every flag but no_graph and staged_loads (which change how a step is
// launched, not what it computes) must match for a bitwise resume.
bool same_flags(const turret_flags &a, const turret_flags &b) {
    turret_flags x = a, y = b;
    x.no_graph = y.no_graph = 0;
    x.staged_loads = y.staged_loads = 0;
    return memcmp(&x, &y, sizeof(turret_flags)) == 0;
}

bool same_config(const CkptHeader &h, const turret_ctx *c) {
    return h.storage == c->storage && h.has_particle == (c->has_particle ? 1 : 0) &&
           h.nm == (c->has_particle ? c->nm : 0) && memcmp(&h.win, &c->win, sizeof(turret_window)) == 0 &&
           same_flags(h.flags, c->flags) && h.nu == c->nu && h.kappa == c->kappa && h.g[0] == c->g[0] &&
           h.g[1] == c->g[1] && h.g[2] == c->g[2] && h.nbox == (c->has_particle ? c->box.nbox : 0);
}

void fill_header(CkptHeader &h, const turret_ctx *c) {
    memset(&h, 0, sizeof h);
    memcpy(h.magic, CKPT_MAGIC, 8);
    h.version = 1;
    h.storage = c->storage;
    h.has_particle = c->has_particle ? 1 : 0;
    h.nm = c->has_particle ? c->nm : 0;
    h.win = c->win;
    h.flags = c->flags;
    h.nu = c->nu;
    h.kappa = c->kappa;
    for (int a = 0; a < 3; ++a) h.g[a] = c->g[a];
    h.step = c->step;
    h.nbox = c->has_particle ? c->box.nbox : 0;
    h.bytes_pop = 27 * c->geom.ncell * (int64_t)storage_bytes(c->storage);
    h.bytes_utop = 3 * c->geom.plane * 4;
    h.bytes_state = sizeof(DevState);
    h.bytes_h = 3 * h.nbox * 4;
    h.bytes_hl = 3 * (int64_t)h.nm * 4;
}
}  // namespace

extern "C" turret_status turret_save(turret_ctx *c, const char *path) {
    if (!c || !path) return fail(c, TURRET_EINVAL, "NULL argument");
    CkptHeader h;
    fill_header(h, c);
    const int p = (int)(c->step & 1);
    struct Part {
        const void *dev;
        int64_t bytes;
    } parts[5] = {{c->f[p], h.bytes_pop},
                  {c->utop[1 - p], h.bytes_utop},
                  {c->dstate, h.bytes_state},
                  {c->has_particle ? c->ba.h : nullptr, h.bytes_h},
                  {c->has_particle ? c->mk.hl : nullptr, h.bytes_hl}};
    CK(cudaStreamSynchronize(c->stream), "save sync");
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(c, TURRET_EINVAL, std::string("cannot open ") + path);
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1;
    std::vector<char> buf;
    for (const Part &q : parts) {
        if (!ok || q.bytes == 0) continue;
        buf.resize((size_t)q.bytes);
        if (cudaMemcpy(buf.data(), q.dev, (size_t)q.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            fclose(fp);
            return cuda_fail(c, cudaGetLastError(), "save copy");
        }
        ok = fwrite(buf.data(), 1, (size_t)q.bytes, fp) == (size_t)q.bytes;
    }
    ok = (fclose(fp) == 0) && ok;
    if (!ok) return fail(c, TURRET_EINVAL, std::string("write failed: ") + path);
    return TURRET_OK;
}

extern "C" turret_status turret_load(turret_ctx *c, const char *path) {
    if (!c || !path) return fail(c, TURRET_EINVAL, "NULL argument");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(c, TURRET_EINVAL, std::string("cannot open ") + path);
    CkptHeader h, want;
    fill_header(want, c);
    if (fread(&h, sizeof h, 1, fp) != 1 || memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != 1) {
        fclose(fp);
        return fail(c, TURRET_EINVAL, "not a checkpoint of this format");
    }
    // every part is copied into the caller's workspace: all five sizes must be
    // the ones this context carves, or a foreign file would overwrite its
    // neighbours
    if (!same_config(h, c) || h.bytes_pop != want.bytes_pop || h.bytes_utop != want.bytes_utop ||
        h.bytes_state != want.bytes_state || h.bytes_h != want.bytes_h || h.bytes_hl != want.bytes_hl) {
        fclose(fp);
        return fail(c, TURRET_ESTATE, "checkpoint of a differently configured context");
    }
    CK(cudaStreamSynchronize(c->stream), "load sync");
    const int p = (int)(h.step & 1);
    void *dst[5] = {c->f[p], c->utop[1 - p], c->dstate, c->has_particle ? c->ba.h : nullptr,
                    c->has_particle ? c->mk.hl : nullptr};
    const int64_t bytes[5] = {h.bytes_pop, h.bytes_utop, h.bytes_state, h.bytes_h, h.bytes_hl};
    std::vector<char> buf;
    for (int k = 0; k < 5; ++k) {
        if (bytes[k] == 0) continue;
        buf.resize((size_t)bytes[k]);
        if (fread(buf.data(), 1, (size_t)bytes[k], fp) != (size_t)bytes[k]) {
            fclose(fp);
            return fail(c, TURRET_EINVAL, "truncated checkpoint");
        }
        if (cudaMemcpy(dst[k], buf.data(), (size_t)bytes[k], cudaMemcpyHostToDevice) != cudaSuccess) {
            fclose(fp);
            return cuda_fail(c, cudaGetLastError(), "load copy");
        }
    }
    fclose(fp);
    c->step = h.step;
    drop_graphs(c);
    return TURRET_OK;
}

extern "C" turret_status lbm_destroy(turret_ctx *c) {
    if (!c) return TURRET_EINVAL;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->aux) cudaStreamSynchronize(c->aux);
    release(c);
    return TURRET_OK;
}

extern "C" const char *turret_last_error(const turret_ctx *c) { return c ? c->err.c_str() : g_init_err.c_str(); }
