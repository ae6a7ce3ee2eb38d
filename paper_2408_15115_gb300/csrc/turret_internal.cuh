// turret_internal.cuh -- device-side data layout shared by the kernels of
// libturret.so (not part of the public ABI).
//
// HBM layout
//   populations : two buffers (ping-pong) of 27 planes [i][z_phys][y][x], each
//                 holding deviations q_i = f_i - w_i in the storage type;
//                 z_phys = (z_logical + ring) mod nz (ring-buffer window).
//   utop        : two buffers [3][ny][nx] float, velocity of the top plane at
//                 the last two collisions (constant-pressure ghost).
//   DevState    : the FP64 rigid-body state and window bookkeeping.
//   support box : a fixed-size block of Bx*By*Bz cells around the particle
//                 (every marker's 4x4x4 Peskin stencil lies inside it), with
//                 u*, sigma and the spread force h as SoA float planes.
//   markers     : SoA arrays, one entry per surface vertex.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace turret {

enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_PRESSURE = 2 };
enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
enum { STAT_OK = 0, STAT_DIVERGED = 5, STAT_DOMAIN = 7 };

// Rigid body + window state, FP64 (Sec. 2.3), resident in device memory.
struct DevState {
    double r[3];       // centre of mass, global coordinates
    double d[9];       // rows d_0, d_1, d_2 of the orientation matrix M
    double v[3], w[3]; // at t - 1/2
    double L[3];       // angular momentum at t - 1/2
    double F[3], T[3]; // hydrodynamic force / torque at t
    double Cf[3];      // centre in window coordinates minus Ci
    long long origin[3];
    long long step;
    int Ci[3];         // floor of the centre in window coordinates
    int box_lo[3];     // window coordinates of support-box cell (0,0,0), unwrapped
    int ring;          // physical plane of logical z = 0
    int reseed_plane;  // physical plane to reset to rest (-1: none)
    int status;
    unsigned int counter;  // last-block ticket of the force reduction
};

// Constant per-context parameters of the fluid window.
struct Geom {
    int nx, ny, nz;
    int bc_x, bc_y, bc_bottom, bc_top;
    int sponge;
    long long plane;  // nx * ny
    long long ncell;  // nx * ny * nz  (population stride)
    float tau0;
    int force_scheme;
};

struct BoxGeom {
    int Bx, By, Bz;
    int tx, ty, tz;   // tiles of 8^3 along each axis
    long long nbox;   // Bx * By * Bz
};

// Rigid-body constants (body frame) and readings.
struct BodyConst {
    double vol, kappa, mass;
    double Jinv_b[9];  // inverse of J/m in the body frame
    double g_eff[3];
    double anchor_z;   // window z the centre is kept near
    int rot_form, renorm, slide;
    int nm;            // markers
    int rc;            // ceil of the bounding radius of the markers about C_m
};

struct MarkerArrays {
    const float *Xb;   // [3][nm] body-frame offsets from C_m
    const float *nb;   // [3][nm] body-frame normals
    const float *dS;   // [nm]
    int *bb;           // [3][nm] stencil base (cell of weight index 0) in box coordinates
    float *wgt;        // [12][nm] Peskin weights along x (4), y (4), z (4)
    float *U;          // [3][nm] prescribed velocity
    float *n;          // [3][nm] lab-frame normal
    float *arm;        // [3][nm] X_k - C_m
    float *hl;         // [3][nm] Lagrangian IBM force
    float *ft;         // [6][nm] dS sigma.n and arm x (dS sigma.n)
};

struct BoxArrays {
    float *u;   // [3][nbox] u*
    float *s;   // [6][nbox] sigma xx yy zz xy xz yz
    float *h;   // [3][nbox] spread force (h_imm after the last cycle)
};

// ---------------------------------------------------------------------------
// D3Q27 index i = ex + 3 ey + 9 ez with e = xi + 1 in {0,1,2}; opposite 26 - i.
// Tensor-product weights w = w1(x) w1(y) w1(z), w1 = (1/6, 2/3, 1/6).
__host__ __device__ constexpr float w1f(int e) { return e == 1 ? (2.0f / 3.0f) : (1.0f / 6.0f); }
__host__ __device__ constexpr float wq(int i) { return w1f(i % 3) * w1f((i / 3) % 3) * w1f(i / 9); }

// Storage codec for the deviation q_i (FP32 arithmetic in every case).
template <int ST> struct Codec;
template <> struct Codec<ST_F32> {
    using T = float;
    static __device__ __forceinline__ float load(const T *p, int) { return __ldg(p); }
    static __device__ __forceinline__ void store(T *p, float q, int) { *p = q; }
};
// FP16: q * 16 / w_i keeps corner populations (w = 1/216) out of subnormals.
template <> struct Codec<ST_F16> {
    using T = __half;
    static __device__ __forceinline__ float load(const T *p, int i) {
        return __half2float(__ldg(p)) * (wq(i) * 0.0625f);
    }
    static __device__ __forceinline__ void store(T *p, float q, int i) {
        *p = __float2half_rn(q * (16.0f / wq(i)));
    }
};
template <> struct Codec<ST_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float load(const T *p, int i) {
        return __bfloat162float(__ldg(p)) * wq(i);
    }
    static __device__ __forceinline__ void store(T *p, float q, int i) {
        *p = __float2bfloat16_rn(q * (1.0f / wq(i)));
    }
};

inline size_t storage_bytes(int st) { return st == ST_F32 ? 4 : 2; }

// ---------------------------------------------------------------------------
// Launchers (lbm_kernels.cu).
cudaError_t launch_collide_stream(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                  float *utop_out, const DevState *st, const float *hbox, const BoxGeom &box,
                                  bool has_box, cudaStream_t s);
cudaError_t launch_init_equilibrium(const Geom &g, int storage, void *dst, const double *drho, const double *u,
                                    float *utop, cudaStream_t s);
cudaError_t launch_macro(const Geom &g, int storage, const void *src, const float *utop_in, const DevState *st,
                         float *out, bool pops, cudaStream_t s);
cudaError_t launch_reseed(const Geom &g, int storage, void *dst, const DevState *st, cudaStream_t s);
cudaError_t launch_box_moments(const Geom &g, int storage, const void *src, const float *utop_in,
                               const DevState *st, const BoxGeom &box, BoxArrays ba, cudaStream_t s);

// Launchers (ibm_kernels.cu).
cudaError_t launch_particle(const Geom &g, const BodyConst &bc, DevState *st, cudaStream_t s);
cudaError_t launch_markers(const Geom &g, const BodyConst &bc, const BoxGeom &box, DevState *st, MarkerArrays m,
                           cudaStream_t s);
cudaError_t launch_bin(const BoxGeom &box, int nm, const int *bb, int *tile_list, int *tile_count, int cap,
                       cudaStream_t s);
cudaError_t launch_interp(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, int mode, cudaStream_t s);
cudaError_t launch_reduce_ft(int nm, MarkerArrays m, double *partials, DevState *st, cudaStream_t s);
cudaError_t launch_spread(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, const int *tile_list,
                          const int *tile_count, int cap, cudaStream_t s);

constexpr int REDUCE_BLOCKS = 32;

}  // namespace turret
