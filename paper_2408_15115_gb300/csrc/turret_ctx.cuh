// turret_ctx.cuh -- the context behind the opaque turret_ctx handle of the
// C ABI (include/turret.h), shared by the single-run and the batch entry points.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/turret.h"
#include "turret_internal.cuh"

struct turret_ctx {
    turret_window win;
    turret_flags flags;
    int storage;
    double nu, tau0, kappa, g[3];
    cudaStream_t stream;  // caller's stream
    cudaStream_t side;    // internal high-priority stream of the immersed-boundary chain
    cudaStream_t aux;     // internal stream of the FP64 force/torque reduction
    cudaEvent_t ev_fork, ev_join, ev_red, ev_red_done, ev_pred;
    // cross-step events of multi-step graphs, by step parity
    cudaEvent_t ev_far[2], ev_near[2], ev_pm[2], ev_ired[2], ev_redd[2], ev_spread[2];
    turret::Geom geom;
    // fluid workspace
    void *f[2];
    // tensor maps of the two population buffers for the staged 16-bit
    // collide+stream: source boxes (lmap) and destination boxes (smap);
    // staged: they were encoded
    CUtensorMap lmap[2], smap[2];
    bool staged;
    float *utop[2];
    turret::DevState *dstate;
    // particle
    bool has_particle;
    bool split;  // near/far collide+stream with the chain on the side stream
    int nm;
    turret::BodyConst body;
    turret::BoxGeom box;
    turret::MarkerArrays mk;
    turret::BoxArrays ba;
    int *tile_list, *tile_count;
    int cap;
    double vol, area;
    turret::DevState host_state;
    turret::DevState *pinned;  // page-locked staging of the device state for queries
    std::vector<float> staging;
    std::vector<float> tau_host;  // staging of the per-plane relaxation times
    // force/torque predictor (surrogate modes) and trajectory log
    int pred_mode, pred_opts;
    float pred_eps;
    double pred_theta;
    const turret_mlp *net;
    double *log;
    long long log_cap;
    // re-injection copy (Sec. 2.5) instead of the ring window; trigger 0 = off
    turret::Reinject reinject;
    // stepping
    long long step;
    cudaGraphExec_t graph[2];
    bool graph_ready[2];
    cudaGraphExec_t graph_multi[2];  // PIPE_STEPS steps per replay, by starting parity
    bool multi_ready[2];
    std::string err;
};

