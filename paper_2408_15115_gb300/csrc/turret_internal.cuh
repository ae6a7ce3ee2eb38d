// turret_internal.cuh -- device-side data layout shared by the kernels of
// libturret.so (not part of the public ABI).
//
// HBM layout
//   populations : two buffers (ping-pong) of 27 planes [i][z_phys][y][x], each
//                 holding scaled deviations s_i = 216 (f_i - w_i) in the
//                 storage type (see Codec below);
//                 z_phys = (z_logical + ring) mod nz (ring-buffer window).
//   utop        : two buffers [3][ny][nx] float, velocity of the top plane at
//                 the last two collisions (constant-pressure ghost).
//   DevState    : the FP64 rigid-body state and window bookkeeping.
//   support box : a fixed-size block of Bx*By*Bz cells around the particle
//                 (every marker's 4x4x4 Peskin stencil lies inside it), with
//                 u*, sigma and the spread force h as SoA float planes.
//   markers     : SoA arrays, one entry per surface vertex.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace turret {

enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_PRESSURE = 2, BC_MOVING = 3 };
enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
enum { STAT_OK = 0, STAT_DIVERGED = 5, STAT_TIMEOUT = 6, STAT_DOMAIN = 7, STAT_OVERFLOW = 8 };

// Rigid body + window state, FP64 (Sec. 2.3), resident in device memory.
// Everything that changes from one time level to the next lives in two slots
// indexed by the parity of the time level t.  Slot t%2 holds the body at t
// (r, d at t; v, w, L at t - 1/2) and the window bookkeeping for pulling f(t)
// from f*(t-1) and for h_imm(t) (ring offset, support-box origin, entering
// plane).  The particle update t -> t+1 reads slot t%2 and writes slot
// (t+1)%2, so collide+stream (reading slot t%2) can run concurrently, and
// every block of the update may recompute it redundantly without racing.
struct BodySlot {
    double r[3];       // centre of mass, global coordinates
    double d[9];       // rows d_0, d_1, d_2 of the orientation matrix M
    double v[3], w[3]; // at t - 1/2
    double L[3];       // angular momentum at t - 1/2
    double Cf[3];      // centre in window coordinates minus Ci
    long long origin[3];
    long long step;
    int Ci[3];         // floor of the centre in window coordinates
    int box_lo[3];     // window coordinates of support-box cell (0,0,0), unwrapped
    int box_lo_w[3];   // the same wrapped into [0, n) along periodic axes
    int ring;          // physical plane of logical z = 0
    int reseed;        // physical plane that entered the ring (reads as rest), -1 none
};

// Force/torque predictor state (surrogate modes; not in the paper).  The
// history is kept in every mode; the prediction is made at the start of a
// step t -> t+1 for F(t+1), T(t+1).
struct Predictor {
    double Fh[4][3], Th[4][3];  // lab-frame F, T at t, t-1, t-2, t-3 (newest first)
    double Fhat[3], That[3];    // prediction for the next time level (the one used)
    double Fnet[3], Tnet[3];    // the network's prediction (made whenever it can run)
    double resid;               // |F - Fhat| / |F| of the last checked prediction
    double resid_net;           // |F - Fnet| / |F| of the network's last prediction
    double ema_net, ema_lin;    // running means (weight 1/8) of the network's and of linear extrapolation's error
    unsigned int slip[8];       // per IBM cycle: max over markers of |U - I[u* + S h]| (float bits)
    int hist_n;                 // valid history entries, 0..4
    int fallback;               // 1: the next prediction is the linear one
    int predicted;              // 1: Fhat, That hold the prediction for the current step
    int by_net;                 // 1: that prediction came from the network
    int net_ok;                 // 1: Fnet, Tnet hold the network's prediction for the current step
    int pad1;
    long long steps, mlp_steps, fallbacks, cycles;  // predictions made, by the network, fallbacks, IBM cycles run
    long long logged;           // trajectory records written
    float feat[40];             // features of the last network prediction (34 used)
    float yb[8];                // its outputs (6 used)
};

struct DevState {
    BodySlot s[2];
    double F[3], T[3];     // hydrodynamic force / torque at the latest time level
    double Fp[3];          // the pressure part of F (F - Fp: viscous part)
    int status;
    unsigned int counter;
    Predictor pr;
};

enum { PRED_WARM = 1, PRED_VEL = 2, PRED_REL = 4 };

// Trajectory record written after the force of each time level j is known:
// d(j) [9], v(j-1/2) [3], w(j-1/2) [3], F(j) [3], T(j) [3], j, |F - Fhat| / |F|
// of the prediction used for j (or -1), Fhat [3], That [3], 1 if the network
// made it (0 linear, -1 none), |F - Fnet| / |F| of the network's prediction
// for j (or -1), 0.
constexpr int LOG_REC = 32;

// Constant per-context parameters of the fluid window.
struct Geom {
    int nx, ny, nz;
    int bc_x, bc_y, bc_bottom, bc_top;
    int sponge;
    long long plane;  // nx * ny
    long long ncell;  // nx * ny * nz  (population stride)
    float tau0;
    int force_scheme;
    int sround;            // 1: BF16 stores round stochastically (counter-based hash)
    float uw_bottom[3], uw_top[3];  // velocities of moving walls (BC_MOVING)
    const float *tau_z;    // [nz] relaxation time per logical plane (sponge included)
    const float *omega_z;  // [nz] 1 / tau per logical plane
};

struct BoxGeom {
    int Bx, By, Bz;
    int tx, ty, tz;   // tiles of TILE^3 along each axis
    long long nbox;   // Bx * By * Bz
};

// Rigid-body constants (body frame) and readings.
struct BodyConst {
    double vol, kappa, mass, inv_mass;
    double Jinv_b[9];  // inverse of J/m in the body frame, divided by the mass
    double g_eff[3];
    double anchor_z;   // window z the centre is kept near
    int rot_form, renorm, slide;
    int fixed;         // 1: the centre is held (v = 0), rotation free
    int force_eval;    // 0: stress on the offset surface (default), 1: at the markers
    int nm;            // markers
    int rc;            // ceil of the bounding radius of the markers about C_m
    float rmin, rmax;  // smallest and largest marker distance from C_m
    // force/torque predictor: 0 the paper's step (marker velocities at
    // t + 1/2, cold IBM cycles); 1 linear extrapolation, 2 network; in modes
    // 1, 2 the marker velocities are predicted at t + 1 and the IBM cycles
    // start from the previous h and stop once the slip is below slip_eps
    int predictor;
    int pred_opts;       // PRED_WARM: warm-started adaptive cycles; PRED_VEL: marker velocities at t + 1;
                         // PRED_REL: resid_theta is relative to linear extrapolation's error
    float slip_eps;
    double resid_theta;  // fall back to the linear prediction above this relative error
    double *log;         // trajectory records [log_cap][LOG_REC], or null
    long long log_cap;
};

// Per-marker record read by the transfer kernels (64 bytes, one per marker):
// packed stencil base in support-box coordinates (x | y << 10 | z << 20), the
// 12 one-dimensional Peskin weights (x0..3, y0..3, z0..3) and h_k dS_k.
// Markers are processed in segments of MARKER_SEG consecutive markers (one
// block of the marker kernel); each segment's stencil bases have a bounding box.
constexpr int MARKER_SEG = 128;
// Offset (cells, along the outward normal) of the surface on which the stress
// is integrated: the kernel half-width, so its stencils lie outside the
// diffuse interface.
constexpr float F_OFFSET = 2.0f;

struct __align__(16) MRec {
    int base;
    float wx[4], wy[4], wz[4];
    float hdS[3];
};

struct MarkerArrays {
    const float *Xb;   // [3][nm] body-frame offsets from C_m
    const float *nb;   // [3][nm] body-frame normals
    const float *dS;   // [nm]
    const float *dSo;  // [nm] areas of the offset surface Xb + F_OFFSET nb (force evaluation)
    MRec *rec;         // [nm] stencil records
    MRec *reco;        // [nm] stencils of the offset points X + F_OFFSET n (stress interpolation)
    int *base;         // [nm] packed stencil bases (copy of rec[k].base, coalesced for binning)
    float *ft;         // [9][nm] dS sigma.n, its moment about C_m, and the pressure part -dS p n
    float *U;          // [3][nm] prescribed velocity
    float *n;          // [3][nm] lab-frame normal
    float *arm;        // [3][nm] X_k - C_m
    float *hl;         // [3][nm] Lagrangian IBM force (the last cycle's result)
    float *r0;         // [3][nm] U_k - I[u*](X_k): the force of step l = 0
    float *hb;         // [3][nm] second buffer of the cycles
    float *aval;       // [nm][ROWCAP] A_kj = dS_j sum_x W(x - X_k) W(x - X_j)
    int *aidx;         // [nm][ROWCAP] column j of each entry, in marker order
    int *alen;         // [nm] entries per row
    int *seg;          // [ceil(nm / MARKER_SEG)][6] per segment of MARKER_SEG consecutive
                       // markers: min x, y, z then max x, y, z of the stencil bases
    int force_eval;    // 0: stress on the offset surface (reco, dSo), 1: at the markers
};

struct BoxArrays {
    float *u;   // [3][nbox] u*
    float *s;   // [6][nbox] sigma xx yy zz xy xz yz
    float *p;   // [nbox] pressure c_s^2 (rho - 1)
    float *h;   // [3][nbox] spread force (h_imm after the last cycle)
};

// Force/torque surrogate network (mlp.cu): 34 -> 3 x 128 GELU -> 6.
constexpr int MLP_IN = 34, MLP_INP = 48, MLP_H = 128, MLP_OUT = 6, MLP_OUTP = 8, MLP_NPARAM = 38278;
struct MlpDev {
    const float *P;            // FP32 parameters, flat layout W1 b1 W2 b2 W3 b3 W4 b4
    const __nv_bfloat16 *Wb;   // BF16 weights, padded: W1 [128][48], W2, W3 [128][128], W4 [8][128]
    const float *mean_x, *std_x, *mean_y, *std_y;
    int precision;             // 0: BF16 tensor cores, 1: FP32
};

// One run of a batch: everything a batched kernel needs about one context,
// in device memory.  A batched launch covers the (run, block) table of all
// runs; block b belongs to run r when prefix[r] <= b < prefix[r + 1].
struct RunDesc {
    Geom g;
    BodyConst bc;
    BoxGeom box;
    MarkerArrays m;
    BoxArrays ba;
    void *f[2];          // ping-pong population buffers
    float *utop[2];      // top-plane velocity buffers
    DevState *st;
    int *tile_list, *tile_count;
    int storage, cap, nm;
    int split;           // 1: far / near collide+stream, 0: the whole window in the near phase
    int tx;              // collide+stream tile width (threads along x)
    MlpDev mlp;          // the force/torque network (predictor mode 2)
};
enum { PHASE_BULK = 0, PHASE_NEAR = 1, PHASE_BULK16 = 2 };

// Run r of block b of a batched launch (largest r < nruns with prefix[r] <=
// b) by one warp: each pass reads 32 table entries at once and narrows the
// range 32-fold by a ballot, so a table of up to 1024 runs takes two
// dependent loads.
__device__ __forceinline__ int find_run_warp(const int *__restrict__ prefix, int nruns, int b, int lane) {
    int lo = 0, span = nruns;
    while (span > 32) {
        const int stride = (span + 31) / 32;
        const int idx = lo + lane * stride;
        const bool ok = idx < lo + span && __ldg(prefix + idx) <= b;
        const unsigned m = __ballot_sync(0xffffffffu, ok);  // entry 0 of the range always qualifies
        lo += (31 - __clz(m)) * stride;
        span = min(stride, nruns - lo);
    }
    const bool ok = lane < span && __ldg(prefix + lo + lane) <= b;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    return lo + (31 - __clz(m));
}

// The run of this block and the block's index within the run, found by warp
// 0 and shared through shared memory (every thread of the block must call).
__device__ __forceinline__ int block_run(const int *__restrict__ prefix, int nruns, int &local) {
    __shared__ int s_run, s_local;
    if (threadIdx.x < 32) {
        const int r = find_run_warp(prefix, nruns, blockIdx.x, threadIdx.x);
        if (threadIdx.x == 0) {
            s_run = r;
            s_local = blockIdx.x - __ldg(prefix + r);
        }
    }
    __syncthreads();
    local = s_local;
    return s_run;
}
// What a batched collide+stream block needs of its run (staged in shared
// memory by every block in one load per thread; the full RunDesc is larger).
struct CollideDesc {
    Geom g;
    BoxGeom box;
    void *f[2];
    float *utop[2];
    DevState *st;
    const float *hbox;
    int storage, split, tx, tx16;  // tx16: tile width of the 16-bit x-pair bulk launch (bulk16)
};
// h arrays of the IBM cycles, selected per run in batched launches
enum { HSEL_R0 = 0, HSEL_HL = 1, HSEL_HB = 2 };

// ---------------------------------------------------------------------------
// D3Q27 index i = ex + 3 ey + 9 ez with e = xi + 1 in {0,1,2}; opposite 26 - i.
// Tensor-product weights w_i = w1(x) w1(y) w1(z), w1 = (1/6, 2/3, 1/6).
//
// Populations are carried as scaled deviations s_i = 216 (f_i - w_i).  The
// scaled weights W_i = 216 w_i = W1(x) W1(y) W1(z), W1 = (1, 4, 1), are the
// exact integers 1, 4, 16, 64, so every equilibrium is formed without weight
// rounding and the collision conserves mass and momentum to round-off
// (float weights 1/216, 1/54, ... would bias the momentum by ~1e-7 per step).
constexpr float SCALE = 216.0f;
constexpr float INV_SCALE = 1.0f / 216.0f;
__host__ __device__ constexpr float W1(int e) { return e == 1 ? 4.0f : 1.0f; }
__host__ __device__ constexpr float Wq(int i) { return W1(i % 3) * W1((i / 3) % 3) * W1(i / 9); }

// Storage codec.  The kernels work in each type's storage domain, in FP32
// arithmetic:
//   FP32: r_i = s_i, the scaled deviation itself;
//   FP16: r_i = K s_i / W_i with K = 16 = 16 (f_i - w_i) / w_i, which keeps
//         corner populations out of subnormals;
//   BF16: r_i = s_i / W_i (K = 1).
// The weights W_i = W1(x) W1(y) W1(z) are exact integers and separable, so
// the scalings fold into the separable moment passes (weights 1, 4, 1 per
// axis) and into the per-axis factors of the collision: loads and stores
// are plain conversions (RN-even on store).
template <int ST> struct Codec;
template <> struct Codec<ST_F32> {
    using T = float;
    static constexpr bool scaled = false;
    static constexpr float K = 1.0f;
    static __device__ __forceinline__ float load(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void store(T *p, float r) { *p = r; }
};
template <> struct Codec<ST_F16> {
    using T = __half;
    static constexpr bool scaled = true;
    static constexpr float K = 16.0f;
    static __device__ __forceinline__ float load(const T *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store(T *p, float r) { *p = __float2half_rn(r); }
};
template <> struct Codec<ST_BF16> {
    using T = __nv_bfloat16;
    static constexpr bool scaled = true;
    static constexpr float K = 1.0f;
    static __device__ __forceinline__ float load(const T *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void store(T *p, float r) { *p = __float2bfloat16_rn(r); }
};

inline size_t storage_bytes(int st) { return st == ST_F32 ? 4 : 2; }

// ---------------------------------------------------------------------------
// Launchers (lbm_kernels.cu).
// Collide+stream region: all cells, the cells outside the near region around
// the particle, or the near region only.  The near region is the region of
// the marker stencils (where h_imm can be nonzero) grown by NEAR_MARGIN cells;
// the support box reaches F_OFFSET cells beyond the marker stencils (the
// stress is read on the offset surface), so the near region is the support
// box grown by NEAR_GROW cells.  It holds every cell the support-box moments
// pull (they skip the box's outer layer), so they wait for the near launch
// only.
enum { REGION_ALL = 0, REGION_FAR = 1, REGION_NEAR = 2 };
constexpr int NEAR_MARGIN = 2;
constexpr int NEAR_GROW = NEAR_MARGIN - 2;
static_assert(F_OFFSET == 2.0f, "the support box grows by F_OFFSET cells per side");
// slot_out >= 0: the kernel also copies the window slot to slot_out (with no
// entering plane) for a following step that has no particle update.
cudaError_t launch_collide_stream(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                  float *utop_out, DevState *st, int slot, int slot_out, const float *hbox,
                                  const BoxGeom &box, bool has_box, int region, cudaStream_t s);
// The far cells of a coupled step (lbm_far.cu): FP32 storage under a register
// cap that leaves room for the immersed-boundary chain's small blocks; 16-bit
// storages staged in shared memory when the tensor maps lmap / smap of src and
// dst are given (see encode_population_map), else on x-adjacent pairs where
// xpair_eligible, else as launch_collide_stream(..., REGION_FAR).
cudaError_t launch_collide_far(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                               float *utop_out, DevState *st, int slot, const float *hbox, const BoxGeom &box,
                               cudaStream_t s, const CUtensorMap *lmap = nullptr, const CUtensorMap *smap = nullptr);
// 16-bit collide+stream with sources and results staged in shared memory by
// bulk tensor copies (lbm_staged.cu): REGION_FAR or REGION_ALL without
// forcing.  staged_eligible: the window's tiling allows it; lmap / smap: the
// source (box 48 x 4 x 2 x 3) and destination (box 32 x 4 x 2 x 27) tensor
// maps of the buffers (encode_population_map); prepare_staged once per device.
bool staged_eligible(const Geom &g, int storage);
bool encode_population_map(CUtensorMap *map, const void *buf, const Geom &g, bool source);
bool prepare_staged();
bool is_staged_kernel(const void *fn);
// 16-bit collide+stream on x-adjacent cell pairs with 4-byte accesses
// (lbm_xpair.cu): REGION_FAR or REGION_ALL without forcing; xpair_eligible:
// FP16 or round-to-nearest BF16 on a window the 64 x 2 x 2 tiles cover.
bool xpair_eligible(const Geom &g, int storage);
bool is_xpair_kernel(const void *fn);
cudaError_t launch_collide_xpair(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                 float *utop_out, DevState *st, int slot, int slot_out, const float *hbox,
                                 const BoxGeom &box, int region, cudaStream_t s);
cudaError_t launch_collide_staged(const Geom &g, int storage, const CUtensorMap &lmap, const CUtensorMap &smap,
                                  const void *src, void *dst, const float *utop_in, float *utop_out, DevState *st,
                                  int slot, int slot_out, const float *hbox, const BoxGeom &box, int region,
                                  cudaStream_t s);
// Re-injection copy of Sec. 2.5 (windows without slide): once the centre's
// window z in slot `slot` is below trigger, the post-collision planes
// [zf - below, zf + above) (zf its floor, clipped) move up by target - zf
// (staged through the other population buffer) and the slot's origin down.
struct Reinject {
    int trigger, target, below, above;
};
cudaError_t launch_reinject(const Geom &g, int storage, void *buf, void *stage, DevState *st, int slot,
                            const Reinject &rj, cudaStream_t s);
cudaError_t launch_init_equilibrium(const Geom &g, int storage, void *dst, const double *drho, const double *u,
                                    float *utop, cudaStream_t s);
cudaError_t launch_macro(const Geom &g, int storage, const void *src, const float *utop_in, const DevState *st,
                         int slot, float *out, bool pops, cudaStream_t s);
// K1 over one window with a 1-D block of `threads` and tile width tx (timing
// of tile candidates; same cells and arithmetic as launch_collide_stream).
// minb: register-budget variant (2: <= 128 registers, 3: <= 85 registers).
bool valid_tile(int threads, int tx, int minb);
cudaError_t launch_collide_tiled(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                 float *utop_out, const DevState *st, int slot, const float *hbox,
                                 const BoxGeom &box, bool has_box, int threads, int tx, int minb, cudaStream_t s);
// Batched K1 of phase PHASE_BULK, PHASE_NEAR or PHASE_BULK16 over nblocks
// blocks (PHASE_BULK16: the far cells of 16-bit runs on x-adjacent pairs,
// 128-thread blocks; threads and minb are ignored).
cudaError_t launch_batch_collide(int phase, const CollideDesc *runs, const int *prefix, int nruns, int p,
                                 int nblocks, int threads, int minb, cudaStream_t s);
bool is_batch_bulk_kernel(const void *fn);
cudaError_t launch_batch_box_moments_bin(const RunDesc *runs, const int *prefix, int nruns, int p, int nblocks,
                                         cudaStream_t s);
// Support-box moments (u*, sigma) and the tile candidate lists, one launch.
// Tiles that no marker can reach (outside the shell rmin <= |X - C_m| <= rmax
// grown by the stencil reach) get empty lists without a scan.
cudaError_t launch_box_moments_bin(const Geom &g, int storage, const void *src, const float *utop_in,
                                   const DevState *st, int slot, const BoxGeom &box, BoxArrays ba, int nm,
                                   const int *mbase, const int *mseg, int *tile_list, int *tile_count, int cap,
                                   DevState *stw, float rmin, float rmax, cudaStream_t s);

// Launchers (ibm_kernels.cu).
// Rigid-body update t -> t+1 (advance = 1; reads window slot `slot`, writes
// slot^1) and the marker kinematics for the resulting state, one launch; with
// advance = 0 only the markers of the current state (window slot `slot`).
cudaError_t launch_particle_markers(const Geom &g, const BodyConst &bc, const BoxGeom &box, DevState *st, int slot,
                                    int advance, MarkerArrays m, cudaStream_t s);
// l = 0 interpolation of u* and sigma, the surface traction per marker, and
// the row k of the interaction matrix A (one warp per marker).
cudaError_t launch_interp0(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, const int *tile_list,
                           const int *tile_count, int cap, DevState *st, int warm, cudaStream_t s,
                           bool by_tile = false);
// One IBM cycle in matrix form: h_out = h_in + r0 - A h_in (= steps l = 1..4).
cudaError_t launch_cycle(int nm, MarkerArrays m, const float *h_in, float *h_out, float *h_final, int last,
                         DevState *st, int cyc, int adaptive, float eps, cudaStream_t s);
// F = sum_k f_k, T = sum_k t_k in FP64, fixed order, into the device state.
cudaError_t launch_reduce_ft(int nm, MarkerArrays m, DevState *st, int slot, const BodyConst &bc, cudaStream_t s);
cudaError_t launch_spread(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, const int *tile_list,
                          const int *tile_count, int cap, cudaStream_t s);
// Batched forms of the launches above, one launch over all runs of a batch
// (time level p -> p ^ 1; blocks per run from the per-phase prefix table).
cudaError_t launch_batch_particle_markers(const RunDesc *runs, const int *prefix, int nruns, int p, int nblocks,
                                          cudaStream_t s);
cudaError_t launch_batch_interp0(const RunDesc *runs, const int *prefix, int nruns, int nblocks, int warm,
                                 cudaStream_t s);
cudaError_t launch_batch_cycle(const RunDesc *runs, const int *prefix, int nruns, int nblocks, int sel_in,
                               int sel_out, int sel_final, int last, int cyc, int adaptive, cudaStream_t s);
cudaError_t launch_batch_reduce_ft(const RunDesc *runs, int nruns, int slot, cudaStream_t s);
cudaError_t launch_batch_predict(const RunDesc *runs, int nruns, int slot, cudaStream_t s);
cudaError_t launch_batch_spread(const RunDesc *runs, const int *prefix, int nruns, int nblocks, cudaStream_t s);
// Blocks of one run in each batched phase (host side, same formulas as the kernels).
int blocks_bulk(const RunDesc &r, int threads);
bool bulk16_run(const RunDesc &r);  // far cells in the 16-bit x-pair bulk launch
int bulk16_tile(const RunDesc &r);  // its tile width
int blocks_bulk16(const RunDesc &r);
int blocks_near(const RunDesc &r, int threads);
int blocks_particle_markers(const RunDesc &r);
int blocks_box_moments_bin(const RunDesc &r);
int blocks_interp0(const RunDesc &r);
int blocks_cycle(const RunDesc &r);
int blocks_spread(const RunDesc &r);

// Forward pass of n raw feature rows x [n][34] -> raw outputs y [n][6].
cudaError_t launch_mlp_infer(const MlpDev &w, const float *x, int n, float *y, cudaStream_t s);
// Force/torque prediction at the start of a step from window slot `slot`
// (mode 1 linear, 2 network w; w may be null), single run or every run.
cudaError_t launch_predict(const MlpDev *w, DevState *st, int slot, int mode, cudaStream_t s);

constexpr int TILE = 4;          // support-box tiles of TILE^3 cells (spreading)
constexpr int INTERP_WARPS = 8;  // markers per interpolation block
constexpr int MAX_CANDIDATES = 2048;  // markers listed per support tile
constexpr int ROWCAP = 512;           // entries per row of A

}  // namespace turret

struct turret_mlp;
const turret::MlpDev *mlp_device_view(const turret_mlp *m);
