/*
 * turret_oracle.c -- plain, slow FP64 CPU oracle for one time step of the
 * Palabos Turret method (arXiv 2408.15115).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the correctness reference that the CUDA
 * path is checked against.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product library never does.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes, in the order of Table 1 (Sec. 2.4):
 *   (1) collide every cell with the recursive-regularized rule (Eq. 7 / Eq. 15
 *       with the equilibrium and off-equilibrium terms of Appendix A), then
 *       stream by pull with the boundary conditions of Sec. 2.5;
 *   (2) advance the rigid particle (leap-frog + orientation predictor-corrector,
 *       Sec. 2.3);
 *   (3) evaluate the stress tensor (Eq. 10) at every node, interpolate it with
 *       the Peskin kernel and sum force / torque (Sec. 2.2 end): at the points
 *       X_k + 2 n_k of the offset surface by default (READING, see
 *       force_torque), or at the markers as printed;
 *   (4) run the multi-direct-forcing IBM cycles (Sec. 2.2, steps l = 0..4,
 *       n = 4 cycles) and spread h_imm onto the dense Eulerian field.
 * Fields are dense arrays over the whole window; loops are explicit.  The
 * Hermite tensors H^(n)_i are built index by index from their generic
 * recurrence, and the coefficients a_1^(n) follow the printed recursion of
 * Appendix A.  Readings of points the paper leaves open are marked "READING".
 *
 * Layout: f[((z*ny + y)*nx + x)*27 + i], lattice index
 * i = (xi_x+1) + 3 (xi_y+1) + 9 (xi_z+1), xi in {-1,0,1}^3 (READING of the
 * garbled "k = 0..2" velocity range of Sec. 2.1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 27
static const double CS2 = 1.0 / 3.0; /* c_s^2 in lattice units (Sec. 2.1) */

/* ------------------------------------------------------------------------ */
/* Lattice (Sec. 2.1, Eq. 4).  READING: the paper prints no weights; we use the
 * standard D3Q27 tensor-product weights w = w1(xi_x) w1(xi_y) w1(xi_z) with
 * w1(0) = 2/3, w1(+-1) = 1/6.                                               */
static int g_xi[NQ][3];
static double g_w[NQ];

/* Hermite tensor component H^(n)_{a_1..a_n}(xi) from the generic recurrence
 *   H^(n)_{a_1..a_n} = xi_{a_n} H^(n-1)_{a_1..a_{n-1}}
 *                      - c_s^2 sum_{j<n} delta_{a_j a_n} H^(n-2)_{a without a_j, a_n}. */
static double hermite(int n, const int *a, const int *xi) {
    if (n == 0) return 1.0;
    if (n == 1) return (double)xi[a[0]];
    double v = (double)xi[a[n - 1]] * hermite(n - 1, a, xi);
    for (int j = 0; j < n - 1; ++j) {
        if (a[j] != a[n - 1]) continue;
        int b[8], m = 0;
        for (int k = 0; k < n - 1; ++k)
            if (k != j) b[m++] = a[k];
        v -= CS2 * hermite(n - 2, b, xi);
    }
    return v;
}

/* The higher-order terms of Appendix A, Eqs. (A.1)/(A.2), in print order.
 * Each entry: index string, multiplicity printed in front of it (1 or 2).
 * The order-n prefactor is 1/(2 c_s^6), 1/(4 c_s^8), 1/(4 c_s^10), 1/(8 c_s^12). */
#define NTERM 17
static const char *k_term_idx[NTERM] = {
    "xxy", "xxz", "xyy", "xzz", "yzz", "yyz", "xyz",      /* order 3 */
    "xxyy", "xxzz", "yyzz", "xyzz", "xyyz", "xxyz",        /* order 4 */
    "xxyzz", "xxyyz", "xyyzz",                              /* order 5 */
    "xxyyzz"};                                              /* order 6 */
static const double k_term_mult[NTERM] = {1, 1, 1, 1, 1, 1, 2, 1, 1, 1, 2, 2, 2, 1, 1, 1, 1};
static int g_term_n[NTERM];
static int g_term_a[NTERM][6];
static double g_term_pref[NTERM];
static double g_H2[NQ][3][3];      /* H^(2)_i,ab */
static double g_Ht[NQ][NTERM];     /* H^(n)_i for the listed index strings */
static int g_ready = 0;

static void lattice_init(void) {
    if (g_ready) return;
    const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    for (int i = 0; i < NQ; ++i) {
        int ex = i % 3, ey = (i / 3) % 3, ez = i / 9;
        g_xi[i][0] = ex - 1; g_xi[i][1] = ey - 1; g_xi[i][2] = ez - 1;
        g_w[i] = w1[ex] * w1[ey] * w1[ez];
    }
    for (int t = 0; t < NTERM; ++t) {
        const char *s = k_term_idx[t];
        int n = (int)strlen(s);
        g_term_n[t] = n;
        for (int k = 0; k < n; ++k) g_term_a[t][k] = s[k] - 'x';
        double cs2n = pow(CS2, n);
        g_term_pref[t] = k_term_mult[t] / ((n == 3 ? 2.0 : n == 6 ? 8.0 : 4.0) * cs2n);
    }
    for (int i = 0; i < NQ; ++i) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int ab[2] = {a, b};
                g_H2[i][a][b] = hermite(2, ab, g_xi[i]);
            }
        for (int t = 0; t < NTERM; ++t) g_Ht[i][t] = hermite(g_term_n[t], g_term_a[t], g_xi[i]);
    }
    g_ready = 1;
}

void orc_lattice(int *xi, double *w) {
    lattice_init();
    for (int i = 0; i < NQ; ++i) {
        for (int a = 0; a < 3; ++a) xi[3 * i + a] = g_xi[i][a];
        w[i] = g_w[i];
    }
}

/* H^(n) of population i for an arbitrary multi-index (test access). */
double orc_hermite(int i, int n, const int *a) {
    lattice_init();
    return hermite(n, a, g_xi[i]);
}

/* ------------------------------------------------------------------------ */
/* Equilibrium, Appendix A Eq. (A.1):
 *   f0_i = w_i (p/c_s^2 + rho_0) ( 1 + xi.u/c_s^2 + H2:uu/(2 c_s^4) + [order 3..6 terms] )
 * with p/c_s^2 + rho_0 = rho (Eq. 5).                                       */
void orc_feq(double rho, const double *u, double *f0) {
    lattice_init();
    double U[NTERM];
    for (int t = 0; t < NTERM; ++t) {
        double p = 1.0;
        for (int k = 0; k < g_term_n[t]; ++k) p *= u[g_term_a[t][k]];
        U[t] = p;
    }
    for (int i = 0; i < NQ; ++i) {
        double s = 1.0;
        s += (g_xi[i][0] * u[0] + g_xi[i][1] * u[1] + g_xi[i][2] * u[2]) / CS2;
        double h2 = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) h2 += g_H2[i][a][b] * u[a] * u[b];
        s += h2 / (2.0 * CS2 * CS2);
        for (int t = 0; t < NTERM; ++t) s += g_term_pref[t] * g_Ht[i][t] * U[t];
        f0[i] = g_w[i] * rho * s;
    }
}

/* Appendix A Eq. (A.3): a_1^(n)_{a1..an} = a_1^(n-1)_{a1..a(n-1)} u_{an}
 *   + ( u_{a1}..u_{a(n-2)} P_{a(n-1) an} + cyclic permutations of a1..a(n-1) ),
 * starting from a_1^(2) = P^(1).  P is the full symmetric 3x3 tensor.        */
static double a1_rec(int n, const int *a, const double *P, const double *u) {
    if (n == 2) return P[3 * a[0] + a[1]];
    double v = a1_rec(n - 1, a, P, u) * u[a[n - 1]];
    /* the n-1 cyclic rotations of (a1..a(n-1)): each index a_j takes the slot
     * paired with a_n once, the others multiply as velocities */
    for (int j = 0; j < n - 1; ++j) {
        double prod = P[3 * a[j] + a[n - 1]];
        for (int k = 0; k < n - 1; ++k)
            if (k != j) prod *= u[a[k]];
        v += prod;
    }
    return v;
}

double orc_a1(int n, const int *a, const double *P, const double *u) { return a1_rec(n, a, P, u); }

/* Off-equilibrium part, Appendix A Eq. (A.2), with P^(1) given (row-major 3x3). */
void orc_fone(const double *P, const double *u, double *f1) {
    lattice_init();
    double A[NTERM];
    for (int t = 0; t < NTERM; ++t) A[t] = a1_rec(g_term_n[t], g_term_a[t], P, u);
    for (int i = 0; i < NQ; ++i) {
        double h2 = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) h2 += g_H2[i][a][b] * P[3 * a + b];
        double s = h2 / (2.0 * CS2 * CS2);
        for (int t = 0; t < NTERM; ++t) s += g_term_pref[t] * g_Ht[i][t] * A[t];
        f1[i] = g_w[i] * s;
    }
}

/* Macroscopic moments, Eq. (5)-(6): rho = sum f, u = sum xi f / sum f, and
 * P^(1) = sum xi xi (f - f0(rho,u))  (Appendix A).                          */
void orc_moments(const double *f, double *rho_out, double *u, double *P) {
    lattice_init();
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < NQ; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += g_xi[i][a] * f[i];
    }
    for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
    double f0[NQ];
    orc_feq(rho, u, f0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int i = 0; i < NQ; ++i) s += g_xi[i][a] * g_xi[i][b] * (f[i] - f0[i]);
            P[3 * a + b] = s;
        }
    *rho_out = rho;
}

/* One cell collision.  force_scheme 0 (READING, default): the regularized form
 * of the equilibrium-velocity shift the paper cites (Shan 2006) applied to
 * f = f0 + f1 with BGK relaxation,
 *     f* = (1-1/tau) f0(rho,u) + (1/tau) f0(rho, u + tau h) + (1-1/tau) f1,
 * which adds exactly rho h of momentum per step and reduces to Eq. (7) at h=0.
 * force_scheme 1: Eq. (15) as printed, f* = f0(rho, u + tau h) + (1-1/tau) f1. */
void orc_collide_cell(const double *f, const double *h, double tau, int force_scheme, double *fout) {
    double rho, u[3], P[9];
    orc_moments(f, &rho, u, P);
    double f0[NQ], f1[NQ], fs[NQ];
    orc_feq(rho, u, f0);
    orc_fone(P, u, f1);
    double us[3] = {u[0] + tau * h[0], u[1] + tau * h[1], u[2] + tau * h[2]};
    orc_feq(rho, us, fs);
    const double om = 1.0 / tau;
    for (int i = 0; i < NQ; ++i) {
        if (force_scheme == 1)
            fout[i] = fs[i] + (1.0 - om) * f1[i];
        else
            fout[i] = (1.0 - om) * f0[i] + om * fs[i] + (1.0 - om) * f1[i];
    }
}

/* Stress tensor, Eq. (10): sigma = -p I + (1/(2 tau) - 1) sum xi xi (f - f0),
 * p = c_s^2 (rho - rho_0) (Eq. 5), f0 at the unforced velocity (READING).   */
void orc_stress(const double *f, double tau, double *sigma, double *u_out) {
    double rho, u[3], P[9];
    orc_moments(f, &rho, u, P);
    const double p = CS2 * (rho - 1.0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) sigma[3 * a + b] = (a == b ? -p : 0.0) + (0.5 / tau - 1.0) * P[3 * a + b];
    if (u_out)
        for (int a = 0; a < 3; ++a) u_out[a] = u[a];
}

/* ------------------------------------------------------------------------ */
/* Peskin 4-point kernel, Sec. 2.2:
 *   w(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8        |r| <= 1
 *        = (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8       1 <= |r| <= 2
 *        = 0 otherwise.                                                     */
double orc_peskin(double r) {
    double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(fmax(0.0, -7.0 + 12.0 * a - 4.0 * a * a))) / 8.0;
    return 0.0;
}

static int cmp64(const void *p, const void *q) {
    int64_t a = *(const int64_t *)p, b = *(const int64_t *)q;
    return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------ */
/* Surface mesh properties (Sec. 2.2 last paragraph and Sec. 2.3).
 *   dS_k: one third of the areas of the triangles sharing vertex k;
 *   n_k : READING, area-weighted mean of the adjacent outward face normals;
 *   V, C_m, J/m: READING of the garbled "J/m = int |x|^2": the inertia tensor
 *        per unit mass about C_m, (1/V) int_V (|x|^2 I - x x^T) dV, by the
 *        divergence theorem (each triangle closes a tetrahedron with the
 *        origin; second moments of a tetrahedron (0,a,b,c) of signed volume v:
 *        int x_i x_j = v/20 (sum_p p_i p_j + s_i s_j), s = a+b+c).
 * Returns 0, or -1 if the mesh is not a closed, consistently oriented
 * two-manifold with positive volume.                                        */
int orc_mesh_props(const double *V, int64_t nv, const int32_t *T, int64_t nt, double *dS, double *nrm,
                   double *vol_out, double *com, double *Jm, double *area_out) {
    /* closedness: every directed edge must appear exactly once and its reverse once */
    int64_t ne = 3 * nt;
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * ne);
    for (int64_t t = 0; t < nt; ++t)
        for (int e = 0; e < 3; ++e) {
            int64_t a = T[3 * t + e], b = T[3 * t + (e + 1) % 3];
            if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) { free(key); return -1; }
            key[3 * t + e] = a * nv + b;
        }
    qsort(key, (size_t)ne, sizeof(int64_t), cmp64);
    int ok = 1;
    for (int64_t k = 1; k < ne; ++k)
        if (key[k] == key[k - 1]) ok = 0;
    for (int64_t k = 0; k < ne && ok; ++k) {
        int64_t a = key[k] / nv, b = key[k] % nv, rk = b * nv + a;
        int64_t lo = 0, hi = ne - 1, found = 0;
        while (lo <= hi) {
            int64_t mid = (lo + hi) / 2;
            if (key[mid] == rk) { found = 1; break; }
            if (key[mid] < rk) lo = mid + 1; else hi = mid - 1;
        }
        if (!found) ok = 0;
    }
    free(key);
    if (!ok) return -1;

    for (int64_t k = 0; k < nv; ++k) {
        dS[k] = 0.0;
        nrm[3 * k] = nrm[3 * k + 1] = nrm[3 * k + 2] = 0.0;
    }
    double vol = 0.0, m1[3] = {0, 0, 0}, m2[9] = {0}, area = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        const double *a = V + 3 * T[3 * t], *b = V + 3 * T[3 * t + 1], *c = V + 3 * T[3 * t + 2];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double ar = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        area += ar;
        for (int e = 0; e < 3; ++e) {
            int64_t k = T[3 * t + e];
            dS[k] += ar / 3.0;
            for (int q = 0; q < 3; ++q) nrm[3 * k + q] += 0.5 * cr[q]; /* area x unit normal */
        }
        double v = (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                    a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
        vol += v;
        double s[3];
        for (int q = 0; q < 3; ++q) {
            s[q] = a[q] + b[q] + c[q];
            m1[q] += v * s[q] / 4.0;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                m2[3 * i + j] += v / 20.0 * (a[i] * a[j] + b[i] * b[j] + c[i] * c[j] + s[i] * s[j]);
    }
    if (!(vol > 0.0)) return -1;
    for (int64_t k = 0; k < nv; ++k) {
        double l = sqrt(nrm[3 * k] * nrm[3 * k] + nrm[3 * k + 1] * nrm[3 * k + 1] + nrm[3 * k + 2] * nrm[3 * k + 2]);
        for (int q = 0; q < 3; ++q) nrm[3 * k + q] /= l;
    }
    for (int q = 0; q < 3; ++q) com[q] = m1[q] / vol;
    /* central second moments S = int (x-c)(x-c)^T = m2 - V c c^T */
    double S[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[3 * i + j] = m2[3 * i + j] - vol * com[i] * com[j];
    double tr = S[0] + S[4] + S[8];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Jm[3 * i + j] = ((i == j ? tr : 0.0) - S[3 * i + j]) / vol;
    *vol_out = vol;
    if (area_out) *area_out = area;
    return 0;
}

/* 3x3 inverse (row-major), by cofactors. */
static void inv3(const double *A, double *B) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    B[0] = c00 / det; B[3] = c01 / det; B[6] = c02 / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

static void cross(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* Simulation object.                                                         */
typedef struct {
    int nx, ny, nz;
    int bc_x, bc_y;           /* 0 periodic, 1 no-slip (halfway bounce-back)     */
    int bc_bottom, bc_top;    /* 0 periodic, 1 no-slip, 2 constant pressure (top),
                               * 3 no-slip wall moving in its plane (uw_*)      */
    int sponge;               /* sponge length in planes below the top            */
    int slide;                /* 1: window follows the particle vertically        */
    double anchor_frac;
    double tau0;              /* tau from nu = c_s^2 (tau - 1/2), Eq. 9           */
    int force_scheme, rot_form, gravity, renorm, ibm_cycles;
    double kappa, g[3];
    int fixed_position;       /* 1: the centre of mass is held (v = 0), rotation free */
    double uw_bottom[3], uw_top[3];  /* velocities of moving walls (bc 3)      */
    /* re-injection copy of Sec. 2.5 (slide = 0; trigger 0 = off): once the
     * centre's window z drops below `trigger`, the planes [zf - below, zf +
     * above) around it (zf = floor of that z) move up by target - zf */
    int reinject_trigger, reinject_target, reinject_below, reinject_above;
    int force_eval;           /* 0: stress on the offset surface X + 2n (READING, default); 1: at the markers */
    /* force/torque predictor (not in the paper; see predict()): 0 the paper's
     * step; 1 linear extrapolation of F, T driving the marker velocities at
     * t + 1; pred_warm 1: the IBM cycles start from the previous step's h and
     * a cycle is skipped once the slip of the previous one is below pred_eps */
    int predictor, pred_warm;
    double pred_eps;
} orc_params;

typedef struct {
    orc_params p;
    int64_t ncell;
    double *f;      /* f(t), pre-collision populations                             */
    double *fpost;  /* f*(t), post-collision                                       */
    double *h;      /* dense h_imm(t), 3 per cell                                  */
    double *u;      /* unforced velocity of f(t), 3 per cell                       */
    double *sig;    /* stress of f(t), 9 per cell                                  */
    double *utop;   /* velocity of the top fluid plane at the last collision       */
    double *tau;    /* relaxation time per plane                                   */
    /* particle */
    int has_particle;
    int64_t nm;
    double *Xb, *nb, *dS;      /* body-frame marker offsets (about C_m), normals, areas */
    double *dSo;               /* areas of the offset surface Xb + OFFSET nb (same triangles) */
    double *X, *n, *U;         /* current window-frame markers, normals, velocities */
    double *hl;                /* Lagrangian IBM force (last h_{l=0} used for h_imm) */
    double vol, Jm[9], Jminv[9], area;
    double r[3], d[9], v[3], w[3], L[3], F[3], T[3];
    double Fp[3];              /* pressure part of F: sum_k dS_k (-p(X_k)) n_k */
    int64_t origin[3], step;
    int status;
    /* predictor state: F, T of the last two force evaluations (newest first),
     * the prediction for the next time level, IBM cycles run */
    double Fh[2][3], Th[2][3], Fhat[3], That[3];
    int hist_n, use_pred, warm_ready;
    int64_t cycles;
} orc_sim;

static inline int64_t cidx(const orc_sim *s, int x, int y, int z) {
    return ((int64_t)z * s->p.ny + y) * s->p.nx + x;
}

/* Sponge (Sec. 2.5): viscosity raised linearly so that tau reaches 1 on the top
 * plane.  READING: tau linear in z over the last `sponge` planes, equal to
 * tau0 on the plane below the sponge and to 1 on the top plane.             */
static void set_tau(orc_sim *s) {
    for (int z = 0; z < s->p.nz; ++z) {
        double t = s->p.tau0;
        int L = s->p.sponge;
        if (L > 0 && z >= s->p.nz - L) t = s->p.tau0 + (1.0 - s->p.tau0) * (double)(z - (s->p.nz - L) + 1) / L;
        s->tau[z] = t;
    }
}

orc_sim *orc_new(const orc_params *p) {
    lattice_init();
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->ncell = (int64_t)p->nx * p->ny * p->nz;
    s->f = (double *)calloc((size_t)s->ncell * NQ, sizeof(double));
    s->fpost = (double *)calloc((size_t)s->ncell * NQ, sizeof(double));
    s->h = (double *)calloc((size_t)s->ncell * 3, sizeof(double));
    s->u = (double *)calloc((size_t)s->ncell * 3, sizeof(double));
    s->sig = (double *)calloc((size_t)s->ncell * 9, sizeof(double));
    s->utop = (double *)calloc((size_t)p->nx * p->ny * 3, sizeof(double));
    s->tau = (double *)calloc((size_t)p->nz, sizeof(double));
    set_tau(s);
    for (int64_t c = 0; c < s->ncell; ++c)
        for (int i = 0; i < NQ; ++i) s->f[c * NQ + i] = s->fpost[c * NQ + i] = g_w[i];
    return s;
}

void orc_free(orc_sim *s) {
    if (!s) return;
    free(s->f); free(s->fpost); free(s->h); free(s->u); free(s->sig); free(s->utop); free(s->tau);
    free(s->Xb); free(s->nb); free(s->dS); free(s->dSo); free(s->X); free(s->n); free(s->U); free(s->hl);
    free(s);
}

/* Moments, velocity and stress of f(t) at every cell. */
static void fields_from_f(orc_sim *s) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cidx(s, x, y, z);
                orc_stress(s->f + c * NQ, s->tau[z], s->sig + 9 * c, s->u + 3 * c);
            }
}

/* Event (1a): collide every cell with h_imm(t). */
static void collide_all(orc_sim *s) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    /* velocity of the top plane at this time level, kept for the pressure ghost */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cidx(s, x, y, z);
                orc_collide_cell(s->f + c * NQ, s->h + 3 * c, s->tau[z], s->p.force_scheme, s->fpost + c * NQ);
                if (z == nz - 1) {
                    double rho, u[3], P[9];
                    orc_moments(s->f + c * NQ, &rho, u, P);
                    for (int a = 0; a < 3; ++a) s->utop[3 * ((int64_t)y * nx + x) + a] = u[a];
                }
            }
}

/* Event (1b): stream by pull, f_i(x, t+1) = f*_i(x - xi_i, t), with
 *   periodic faces: wrap;
 *   no-slip faces (READING: halfway bounce-back, wall half a cell outside the
 *     first/last node): f_i(x) = f*_{opp(i)}(x) when x - xi_i is outside;
 *   constant-pressure top (READING): the ghost node above the top plane holds
 *     f0(rho = 1, u_top) with u_top the velocity of the top fluid node below
 *     the ghost at the previous collision.
 * A source outside a no-slip face takes precedence over the pressure ghost.
 *   moving wall (bc 3, shear flows; READING, the paper gives no rule): the
 *     halfway bounce-back of a wall moving with velocity u_w in its plane adds
 *     the momentum the wall imparts, f_i(x) = f*_{opp i}(x) + 2 w_i rho_w
 *     (xi_i . u_w) / c_s^2 with rho_w = 1 (the reference density), for every
 *     population whose source lies beyond that face.                       */
static void stream_all(orc_sim *s) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cidx(s, x, y, z);
                for (int i = 0; i < NQ; ++i) {
                    int sx = x - g_xi[i][0], sy = y - g_xi[i][1], sz = z - g_xi[i][2];
                    int bb = 0, ghost = 0;
                    const double *uw = NULL;
                    if (sx < 0 || sx >= nx) {
                        if (s->p.bc_x == 1) bb = 1; else sx = (sx + nx) % nx;
                    }
                    if (sy < 0 || sy >= ny) {
                        if (s->p.bc_y == 1) bb = 1; else sy = (sy + ny) % ny;
                    }
                    if (sz < 0) {
                        if (s->p.bc_bottom == 1 || s->p.bc_bottom == 3) bb = 1; else sz = (sz + nz) % nz;
                        if (s->p.bc_bottom == 3) uw = s->p.uw_bottom;
                    } else if (sz >= nz) {
                        if (s->p.bc_top == 1 || s->p.bc_top == 3) bb = 1;
                        else if (s->p.bc_top == 2) ghost = 1;
                        else sz = sz % nz;
                        if (s->p.bc_top == 3) uw = s->p.uw_top;
                    }
                    double val;
                    if (bb) {
                        val = s->fpost[c * NQ + (NQ - 1 - i)];
                        if (uw) val += 6.0 * g_w[i] * (g_xi[i][0] * uw[0] + g_xi[i][1] * uw[1] + g_xi[i][2] * uw[2]);
                    } else if (ghost) {
                        double f0[NQ];
                        orc_feq(1.0, s->utop + 3 * ((int64_t)sy * nx + sx), f0);
                        val = f0[i];
                    } else {
                        val = s->fpost[cidx(s, sx, sy, sz) * NQ + i];
                    }
                    s->f[c * NQ + i] = val;
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Fluid initialisation: the post-collision state f*(-1) is the equilibrium of
 * the given density and velocity fields (rho, u per cell; NULL = rest), the
 * pressure-ghost velocity is the given top-plane velocity, and f(0) follows by
 * one streaming.                                                            */
void orc_init_fields(orc_sim *s, const double *rho, const double *u) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    for (int64_t c = 0; c < s->ncell; ++c) {
        double r = rho ? rho[c] : 1.0;
        double uu[3] = {0, 0, 0};
        if (u) { uu[0] = u[3 * c]; uu[1] = u[3 * c + 1]; uu[2] = u[3 * c + 2]; }
        orc_feq(r, uu, s->fpost + c * NQ);
    }
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int a = 0; a < 3; ++a)
                s->utop[3 * ((int64_t)y * nx + x) + a] = u ? u[3 * cidx(s, x, y, nz - 1) + a] : 0.0;
    stream_all(s);
    memset(s->h, 0, sizeof(double) * 3 * (size_t)s->ncell);
    fields_from_f(s);
    s->step = 0;
}

/* Dense body-force field h (3 per cell) used by the next collisions (fluid-only
 * studies such as Poiseuille). */
void orc_set_force(orc_sim *s, const double *h) { memcpy(s->h, h, sizeof(double) * 3 * (size_t)s->ncell); }

/* One fluid-only step: collide with the current h, stream, refresh fields. */
void orc_fluid_step(orc_sim *s, int n) {
    for (int k = 0; k < n; ++k) {
        collide_all(s);
        stream_all(s);
        fields_from_f(s);
        s->step++;
    }
}

void orc_get_f(const orc_sim *s, double *out) { memcpy(out, s->f, sizeof(double) * NQ * (size_t)s->ncell); }
void orc_get_fpost(const orc_sim *s, double *out) { memcpy(out, s->fpost, sizeof(double) * NQ * (size_t)s->ncell); }
void orc_set_f(orc_sim *s, const double *in) {
    memcpy(s->f, in, sizeof(double) * NQ * (size_t)s->ncell);
    fields_from_f(s);
}
void orc_get_velocity(const orc_sim *s, double *out) { memcpy(out, s->u, sizeof(double) * 3 * (size_t)s->ncell); }
void orc_get_stress(const orc_sim *s, double *out) { memcpy(out, s->sig, sizeof(double) * 9 * (size_t)s->ncell); }
void orc_get_force_field(const orc_sim *s, double *out) { memcpy(out, s->h, sizeof(double) * 3 * (size_t)s->ncell); }
void orc_get_utop(const orc_sim *s, double *out) { memcpy(out, s->utop, sizeof(double) * 3 * (size_t)s->p.nx * s->p.ny); }

/* ------------------------------------------------------------------------ */
/* Eulerian <-> Lagrangian transfer with the Peskin kernel (Sec. 2.2), lattice
 * units (dx = dt = 1).  READING: the paper's W carries 1/dx^3 and the sums
 * carry dx^3 (interpolation) and dS_k (spreading); with dx = 1 these are
 *   I[u](X) = sum_x u(x) w(x-X) w(y-Y) w(z-Z),
 *   S[h](x) = sum_k h_k w(x-X_k) w(y-Y_k) w(z-Z_k) dS_k.
 * The stencil is the 4x4x4 block of cells floor(X)-1 .. floor(X)+2 in each
 * axis (every other cell has zero weight).  Periodic axes wrap.             */
typedef struct {
    int nx, ny, nz, per_x, per_y, per_z;
} orc_grid;

static int wrapc(int c, int n, int per) {
    if (per) return ((c % n) + n) % n;
    return c; /* caller guarantees the stencil is inside non-periodic axes */
}

void orc_interp(const orc_grid *g, const double *field, int ncomp, const double *X, int64_t nm, double *out) {
    for (int64_t k = 0; k < nm; ++k) {
        const double *Xk = X + 3 * k;
        int b[3] = {(int)floor(Xk[0]) - 1, (int)floor(Xk[1]) - 1, (int)floor(Xk[2]) - 1};
        for (int c = 0; c < ncomp; ++c) out[ncomp * k + c] = 0.0;
        for (int dz = 0; dz < 4; ++dz)
            for (int dy = 0; dy < 4; ++dy)
                for (int dx = 0; dx < 4; ++dx) {
                    int x = b[0] + dx, y = b[1] + dy, z = b[2] + dz;
                    double W = orc_peskin(x - Xk[0]) * orc_peskin(y - Xk[1]) * orc_peskin(z - Xk[2]);
                    int64_t cell = ((int64_t)wrapc(z, g->nz, g->per_z) * g->ny + wrapc(y, g->ny, g->per_y)) * g->nx +
                                   wrapc(x, g->nx, g->per_x);
                    for (int c = 0; c < ncomp; ++c) out[ncomp * k + c] += field[ncomp * cell + c] * W;
                }
    }
}

void orc_spread(const orc_grid *g, const double *hk, const double *X, const double *dS, int64_t nm, double *field) {
    int64_t ncell = (int64_t)g->nx * g->ny * g->nz;
    memset(field, 0, sizeof(double) * 3 * (size_t)ncell);
    for (int64_t k = 0; k < nm; ++k) {
        const double *Xk = X + 3 * k;
        int b[3] = {(int)floor(Xk[0]) - 1, (int)floor(Xk[1]) - 1, (int)floor(Xk[2]) - 1};
        for (int dz = 0; dz < 4; ++dz)
            for (int dy = 0; dy < 4; ++dy)
                for (int dx = 0; dx < 4; ++dx) {
                    int x = b[0] + dx, y = b[1] + dy, z = b[2] + dz;
                    double W = orc_peskin(x - Xk[0]) * orc_peskin(y - Xk[1]) * orc_peskin(z - Xk[2]);
                    int64_t cell = ((int64_t)wrapc(z, g->nz, g->per_z) * g->ny + wrapc(y, g->ny, g->per_y)) * g->nx +
                                   wrapc(x, g->nx, g->per_x);
                    for (int c = 0; c < 3; ++c) field[3 * cell + c] += hk[3 * k + c] * W * dS[k];
                }
    }
}

/* Multi-direct forcing, Sec. 2.2, steps l = 0..4 repeated for n cycles:
 *   l=0: h0_k = (U_k - I[u*](X_k)) / dt
 *   l=1: h1(x) = S[h0](x)
 *   l=2: u2(x) = u*(x) + h1(x) dt
 *   l=3: u3_k = I[u2](X_k)
 *   l=4: h0_k <- h0_k + (U_k - u3_k) / dt, next cycle from l=1.
 * h_imm is h1 of the last cycle, so steps l=2..4 of the last cycle are not
 * run.  Outputs: himm (dense, 3 per cell) and hl (the Lagrangian force that
 * was spread, 3 per marker).                                                 */
/* The IBM cycles warm-started from a given Lagrangian force h (predictor
 * option, not in the paper): for cycle 1 .. ncycles, unless the previous
 * cycle's slip max_k |U_k - I[u* + S h](X_k)| (over markers and components)
 * is below eps, h <- h + U - I[u* + S h]; then h_imm = S[h].  hl: h on entry
 * and on return.  Returns the cycles run.                                    */
int orc_ibm_warm(const orc_grid *g, const double *ustar, const double *X, const double *U, const double *dS, int64_t nm,
                 int ncycles, double eps, double *himm, double *hl) {
    int64_t ncell = (int64_t)g->nx * g->ny * g->nz;
    double *ui = (double *)malloc(sizeof(double) * 3 * (size_t)nm);
    double *u2 = (double *)malloc(sizeof(double) * 3 * (size_t)ncell);
    double slip = INFINITY;
    int run = 0;
    for (int cyc = 1; cyc <= ncycles; ++cyc) {
        if (cyc > 1 && slip < eps) break;
        orc_spread(g, hl, X, dS, nm, himm);
        for (int64_t c = 0; c < 3 * ncell; ++c) u2[c] = ustar[c] + himm[c];
        orc_interp(g, u2, 3, X, nm, ui);
        slip = 0.0;
        for (int64_t k = 0; k < 3 * nm; ++k) {
            const double r = U[k] - ui[k];
            if (fabs(r) > slip) slip = fabs(r);
            hl[k] += r;
        }
        run += 1;
    }
    orc_spread(g, hl, X, dS, nm, himm);
    free(ui);
    free(u2);
    return run;
}

void orc_ibm(const orc_grid *g, const double *ustar, const double *X, const double *U, const double *dS, int64_t nm,
             int ncycles, double *himm, double *hl) {
    int64_t ncell = (int64_t)g->nx * g->ny * g->nz;
    double *ui = (double *)malloc(sizeof(double) * 3 * (size_t)nm);
    double *u2 = (double *)malloc(sizeof(double) * 3 * (size_t)ncell);
    orc_interp(g, ustar, 3, X, nm, ui);
    for (int64_t k = 0; k < 3 * nm; ++k) hl[k] = U[k] - ui[k];
    for (int cyc = 1; cyc <= ncycles; ++cyc) {
        orc_spread(g, hl, X, dS, nm, himm);
        if (cyc == ncycles) break;
        for (int64_t c = 0; c < 3 * ncell; ++c) u2[c] = ustar[c] + himm[c];
        orc_interp(g, u2, 3, X, nm, ui);
        for (int64_t k = 0; k < 3 * nm; ++k) hl[k] += U[k] - ui[k];
    }
    free(ui);
    free(u2);
}

/* ------------------------------------------------------------------------ */
/* Rigid particle.                                                           */
static orc_grid sim_grid(const orc_sim *s) {
    orc_grid g = {s->p.nx, s->p.ny, s->p.nz, s->p.bc_x == 0, s->p.bc_y == 0,
                  s->p.bc_bottom == 0 && s->p.bc_top == 0};
    return g;
}

/* Marker kinematics, Sec. 2.3: X_k = C + M^T Xb_k (M has rows d_i, so M^T maps
 * body to lab components), n_k = M^T nb_k, U_k = v + omega x (X_k - C), with C
 * the centre of mass in window coordinates (READING: U_k from v, omega at
 * t + dt/2, the only level available at event (4), and X_k at t + dt).      */
static void marker_motion(const orc_sim *s, double vel[3], double om[3]);

static void update_markers(orc_sim *s) {
    double C[3] = {s->r[0] - (double)s->origin[0], s->r[1] - (double)s->origin[1], s->r[2] - (double)s->origin[2]};
    double vel[3], om[3];
    marker_motion(s, vel, om);
    for (int64_t k = 0; k < s->nm; ++k) {
        double arm[3], nn[3];
        for (int a = 0; a < 3; ++a) {
            arm[a] = 0.0;
            nn[a] = 0.0;
            for (int i = 0; i < 3; ++i) {
                arm[a] += s->d[3 * i + a] * s->Xb[3 * k + i];
                nn[a] += s->d[3 * i + a] * s->nb[3 * k + i];
            }
        }
        double wx[3];
        cross(om, arm, wx);
        for (int a = 0; a < 3; ++a) {
            s->X[3 * k + a] = C[a] + arm[a];
            s->n[3 * k + a] = nn[a];
            s->U[3 * k + a] = vel[a] + wx[a];
        }
    }
}

/* Marker stencils must lie inside the window along non-periodic axes
 * (READING: the paper is silent; anything else would read outside). */
/* Distance along the outward normal of the surface on which the stress is
 * evaluated (force_eval 0): the kernel half-width, so that the interpolation
 * stencil of X + OFFSET n lies entirely on the fluid side of the markers. */
#define OFFSET 2.0

static int check_support(const orc_sim *s) {
    orc_grid g = sim_grid(s);
    int per[3] = {g.per_x, g.per_y, g.per_z}, n[3] = {g.nx, g.ny, g.nz};
    const double off = s->p.force_eval == 0 ? OFFSET : 0.0;
    for (int64_t k = 0; k < s->nm; ++k)
        for (int a = 0; a < 3; ++a) {
            if (per[a]) continue;
            int b = (int)floor(s->X[3 * k + a]);
            if (b - 1 < 0 || b + 2 > n[a] - 1) return -2;
            b = (int)floor(s->X[3 * k + a] + off * s->n[3 * k + a]);
            if (b - 1 < 0 || b + 2 > n[a] - 1) return -2;
        }
    return 0;
}

/* Surface force and torque, Sec. 2.2 end:
 *   F = sum_k dS_k sigma(X_k) n_k,  sigma(X_k) = sum_x sigma(x) W(x - X_k),
 *   T = sum_k (X_k - C_m) x (dS_k sigma(X_k) n_k).
 * READING: the printed torque "[sigma n] ^ (X_k - C_m)" is -(r x F); we take
 * the physical moment r x F. rho_f = 1.
 * READING (force_eval 0, default): the IBM fluid fills the body too, and a
 * stencil centred on X_k averages the exterior traction with the interior's
 * (rigid motion: no viscous stress), which was measured 2-3 times too small
 * (a sphere settling at about twice its confined Stokes velocity, a spinning
 * sphere feeling 0.45 of its Stokes torque).  The stress is therefore taken on
 * the offset surface X_k + OFFSET n_k, whose stencils lie on the fluid side,
 * with that surface's areas dSo_k and arms X_k + OFFSET n_k - C_m: for steady
 * Stokes flow the stress integral over any surface enclosing the body is the
 * same, and this one encloses the whole diffuse interface.  force_eval 1: the
 * formula as printed.  Fp: the pressure part -p I of the same integral.      */
static void force_torque(orc_sim *s) {
    orc_grid g = sim_grid(s);
    const int off = s->p.force_eval == 0;
    double *Xs = (double *)malloc(sizeof(double) * 3 * (size_t)s->nm);
    for (int64_t k = 0; k < s->nm; ++k)
        for (int a = 0; a < 3; ++a) Xs[3 * k + a] = s->X[3 * k + a] + (off ? OFFSET * s->n[3 * k + a] : 0.0);
    const double *area = off ? s->dSo : s->dS;
    double *sk = (double *)malloc(sizeof(double) * 9 * (size_t)s->nm);
    orc_interp(&g, s->sig, 9, Xs, s->nm, sk);
    /* the isotropic part of Eq. (10) alone: p = c_s^2 (rho - 1) per cell from
     * the same populations, interpolated likewise; its surface sum is the
     * pressure force, F - Fp the viscous one */
    double *pc = (double *)malloc(sizeof(double) * (size_t)s->ncell);
    for (int64_t c = 0; c < s->ncell; ++c) {
        double rho = 0.0;
        for (int i = 0; i < NQ; ++i) rho += s->f[c * NQ + i];
        pc[c] = (rho - 1.0) / 3.0;
    }
    double *pk = (double *)malloc(sizeof(double) * (size_t)s->nm);
    orc_interp(&g, pc, 1, Xs, s->nm, pk);
    double C[3] = {s->r[0] - (double)s->origin[0], s->r[1] - (double)s->origin[1], s->r[2] - (double)s->origin[2]};
    for (int a = 0; a < 3; ++a) s->F[a] = s->T[a] = s->Fp[a] = 0.0;
    for (int64_t k = 0; k < s->nm; ++k) {
        double fk[3], arm[3], tk[3];
        for (int a = 0; a < 3; ++a) {
            fk[a] = 0.0;
            for (int b = 0; b < 3; ++b) fk[a] += sk[9 * k + 3 * a + b] * s->n[3 * k + b];
            fk[a] *= area[k];
            arm[a] = Xs[3 * k + a] - C[a];
            s->Fp[a] -= area[k] * pk[k] * s->n[3 * k + a];
        }
        cross(arm, fk, tk);
        for (int a = 0; a < 3; ++a) {
            s->F[a] += fk[a];
            s->T[a] += tk[a];
        }
    }
    free(pk);
    free(pc);
    free(sk);
    free(Xs);
}

static void run_ibm(orc_sim *s) {
    orc_grid g = sim_grid(s);
    if (s->p.predictor && s->p.pred_warm && s->warm_ready) {
        s->cycles += orc_ibm_warm(&g, s->u, s->X, s->U, s->dS, s->nm, s->p.ibm_cycles, s->p.pred_eps, s->h, s->hl);
    } else {
        orc_ibm(&g, s->u, s->X, s->U, s->dS, s->nm, s->p.ibm_cycles, s->h, s->hl);
        s->cycles += s->p.ibm_cycles - 1;
    }
    s->warm_ready = 1;  /* every later step may start from this h */
}


/* 6DOF update, Sec. 2.3 (leap-frog, Eqs. 22-27), dt = 1, rho_f = 1, m = kappa V:
 *   a = g_eff + F/(kappa V);  v(t+1/2) = v(t-1/2) + a;  r(t+1) = r(t) + v(t+1/2)
 *   rotation, rot_form 1 (as printed):
 *     omega(t+1/2) = omega(t-1/2) + M^T (J/m)^-1 M T / (kappa V)
 *   rotation, rot_form 0 (READING, default): the printed dw/dt = J^-1 T omits
 *     the gyroscopic term; we advance the angular momentum instead,
 *     L(t+1/2) = L(t-1/2) + T,  omega(t+1/2) = M^T (J/m)^-1 M L / (kappa V);
 *   d_i^pred = d_i + omega x d_i;  d_i(t+1) = d_i + omega x (d_i + d_i^pred)/2.
 * M has rows d_i(t).  g_eff: gravity 1 = g as printed; gravity 0 (READING,
 * default) = (1 - 1/kappa) g, the buoyancy the printed a = g + F/m leaves out
 * because the fluid carries no hydrostatic gradient.                          */
static void advance_particle(orc_sim *s) {
    const double m = s->p.kappa * s->vol;
    double ge[3];
    for (int a = 0; a < 3; ++a) ge[a] = (s->p.gravity == 1 ? 1.0 : 1.0 - 1.0 / s->p.kappa) * s->p.g[a];
    for (int a = 0; a < 3; ++a) {
        double acc = ge[a] + s->F[a] / m;
        s->v[a] = s->p.fixed_position ? 0.0 : s->v[a] + acc;
        s->r[a] += s->v[a];
    }
    double src[3], sb[3], wb[3];
    if (s->p.rot_form == 1) {
        for (int a = 0; a < 3; ++a) src[a] = s->T[a];
    } else {
        for (int a = 0; a < 3; ++a) {
            s->L[a] += s->T[a];
            src[a] = s->L[a];
        }
    }
    for (int i = 0; i < 3; ++i) sb[i] = s->d[3 * i] * src[0] + s->d[3 * i + 1] * src[1] + s->d[3 * i + 2] * src[2];
    for (int i = 0; i < 3; ++i) wb[i] = (s->Jminv[3 * i] * sb[0] + s->Jminv[3 * i + 1] * sb[1] + s->Jminv[3 * i + 2] * sb[2]) / m;
    double wl[3];
    for (int a = 0; a < 3; ++a) wl[a] = s->d[a] * wb[0] + s->d[3 + a] * wb[1] + s->d[6 + a] * wb[2];
    for (int a = 0; a < 3; ++a) s->w[a] = (s->p.rot_form == 1) ? s->w[a] + wl[a] : wl[a];
    double dn[9];
    for (int i = 0; i < 3; ++i) {
        double pred[3], c1[3], mid[3], c2[3];
        cross(s->w, s->d + 3 * i, c1);
        for (int a = 0; a < 3; ++a) pred[a] = s->d[3 * i + a] + c1[a];
        for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (s->d[3 * i + a] + pred[a]);
        cross(s->w, mid, c2);
        for (int a = 0; a < 3; ++a) dn[3 * i + a] = s->d[3 * i + a] + c2[a];
    }
    memcpy(s->d, dn, sizeof dn);
    if (s->p.renorm) { /* modified Gram-Schmidt d0, d1, d2 */
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < i; ++j) {
                double pj = 0.0;
                for (int a = 0; a < 3; ++a) pj += s->d[3 * i + a] * s->d[3 * j + a];
                for (int a = 0; a < 3; ++a) s->d[3 * i + a] -= pj * s->d[3 * j + a];
            }
            double l = sqrt(s->d[3 * i] * s->d[3 * i] + s->d[3 * i + 1] * s->d[3 * i + 1] + s->d[3 * i + 2] * s->d[3 * i + 2]);
            for (int a = 0; a < 3; ++a) s->d[3 * i + a] /= l;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Force/torque predictor.  Not part of the paper, whose only predictor is the
 * orientation predictor-corrector above; the marker velocities of the IBM
 * step (event 4) are otherwise taken at t + 1/2.  With predictor 1 the force
 * and torque of the next time level are extrapolated linearly from the last
 * two evaluations, F^(t+1) = 2 F(t) - F(t-1) (F(t) alone after the first
 * evaluation), and the markers move with the estimate of the body's motion at
 * t + 1 that this gives, half a leap-frog step on from t + 1/2:
 *   v^ = v(t+1/2) + (g_eff + F^ / m) / 2          (0 for a held centre),
 *   angular momentum form: L^ = L(t+1/2) + T^ / 2,  omega^ = M^T (J/m)^-1 M L^ / m,
 *   printed form:  omega^ = omega(t+1/2) + M^T (J/m)^-1 M T^ / (2 m),
 * with M the orientation at t + 1.                                           */
static void push_history(orc_sim *s) {
    for (int a = 0; a < 3; ++a) {
        s->Fh[1][a] = s->Fh[0][a];
        s->Th[1][a] = s->Th[0][a];
        s->Fh[0][a] = s->F[a];
        s->Th[0][a] = s->T[a];
    }
    if (s->hist_n < 2) s->hist_n += 1;
}

static void predict(orc_sim *s) {
    for (int a = 0; a < 3; ++a) {
        s->Fhat[a] = s->hist_n >= 2 ? 2.0 * s->Fh[0][a] - s->Fh[1][a] : s->Fh[0][a];
        s->That[a] = s->hist_n >= 2 ? 2.0 * s->Th[0][a] - s->Th[1][a] : s->Th[0][a];
    }
}

/* Translational and angular velocity the markers move with: v, omega at
 * t + 1/2 (the paper), or the predicted estimates at t + 1. */
static void marker_motion(const orc_sim *s, double vel[3], double om[3]) {
    if (!s->use_pred) {
        for (int a = 0; a < 3; ++a) {
            vel[a] = s->v[a];
            om[a] = s->w[a];
        }
        return;
    }
    const double m = s->p.kappa * s->vol;
    for (int a = 0; a < 3; ++a) {
        const double ge = (s->p.gravity == 1 ? 1.0 : 1.0 - 1.0 / s->p.kappa) * s->p.g[a];
        vel[a] = s->p.fixed_position ? 0.0 : s->v[a] + 0.5 * (ge + s->Fhat[a] / m);
    }
    double src[3], sb[3], wb[3];
    for (int a = 0; a < 3; ++a) src[a] = s->p.rot_form == 1 ? s->That[a] : s->L[a] + 0.5 * s->That[a];
    for (int i = 0; i < 3; ++i) sb[i] = s->d[3 * i] * src[0] + s->d[3 * i + 1] * src[1] + s->d[3 * i + 2] * src[2];
    for (int i = 0; i < 3; ++i) wb[i] = (s->Jminv[3 * i] * sb[0] + s->Jminv[3 * i + 1] * sb[1] + s->Jminv[3 * i + 2] * sb[2]) / m;
    for (int a = 0; a < 3; ++a) {
        const double wl = s->d[a] * wb[0] + s->d[3 + a] * wb[1] + s->d[6 + a] * wb[2];
        om[a] = s->p.rot_form == 1 ? s->w[a] + 0.5 * wl : wl;
    }
}

/* Vertical window slide.  READING of the re-injection copy of Sec. 2.5: the
 * window follows the particle one plane at a time instead of copying a block
 * back; when the centre is one cell or more below (above) its anchor plane
 * anchor_frac * nz, every post-collision plane moves up (down) by one, the
 * entering plane is set to the rest equilibrium and the origin moves.  Done on
 * f*(t), between collision and streaming (events (1) and (2) commute).       */
static void slide_window(orc_sim *s) {
    if (!s->p.slide) return;
    const int nz = s->p.nz;
    const int64_t plane = (int64_t)s->p.nx * s->p.ny * NQ;
    double dz = (s->r[2] - (double)s->origin[2]) - s->p.anchor_frac * nz;
    if (dz <= -1.0) {
        memmove(s->fpost + plane, s->fpost, sizeof(double) * (size_t)(plane * (nz - 1)));
        for (int64_t c = 0; c < plane / NQ; ++c)
            for (int i = 0; i < NQ; ++i) s->fpost[c * NQ + i] = g_w[i];
        s->origin[2] -= 1;
    } else if (dz >= 1.0) {
        memmove(s->fpost, s->fpost + plane, sizeof(double) * (size_t)(plane * (nz - 1)));
        for (int64_t c = 0; c < plane / NQ; ++c)
            for (int i = 0; i < NQ; ++i) s->fpost[plane * (nz - 1) + c * NQ + i] = g_w[i];
        s->origin[2] += 1;
    }
}

/* Re-injection copy, Sec. 2.5, as printed in spirit (READING: the block
 * extents and the jump are parameters; the paper gives ~60% of h, elongated
 * above the particle): when the centre's window z = r_z - origin_z has fallen
 * below the trigger plane, the post-collision planes [zf - below, zf + above)
 * (zf = floor z, clipped to the window) are copied up by dz = target - zf
 * (planes that would leave the top are dropped) and the window origin moves
 * down by dz, so the particle keeps its global position and lands at the
 * target plane.  Fluid outside the copied block is left as it was.  Done on
 * f*(t) after the particle update, like the ring slide.                     */
static void reinject(orc_sim *s) {
    if (s->p.slide || s->p.reinject_trigger <= 0) return;
    const int nz = s->p.nz;
    const double zc = s->r[2] - (double)s->origin[2];
    if (!(zc < (double)s->p.reinject_trigger)) return;
    const int zf = (int)floor(zc);
    const int dz = s->p.reinject_target - zf;
    if (dz <= 0) return;
    int z0 = zf - s->p.reinject_below, z1 = zf + s->p.reinject_above;
    if (z0 < 0) z0 = 0;
    if (z1 > nz - dz) z1 = nz - dz;
    const int64_t plane = (int64_t)s->p.nx * s->p.ny * NQ;
    if (z1 > z0)
        memmove(s->fpost + plane * (z0 + dz), s->fpost + plane * z0, sizeof(double) * (size_t)(plane * (z1 - z0)));
    s->origin[2] -= dz;
}

/* Particle definition.  verts: body mesh (any origin; re-centred on its centre
 * of mass, body frame = lab frame at t = 0), tris: outward CCW triangles.
 * r0: centre of mass in window coordinates at t = 0; v0, w0: v(-1/2),
 * omega(-1/2).  Runs events (3) and (4) once so that F(0), T(0) and h_imm(0)
 * are defined.  Returns 0, -1 for a bad mesh, -2 for markers too close to a
 * non-periodic face.                                                         */
int orc_load_particle(orc_sim *s, const double *verts, int64_t nv, const int32_t *tris, int64_t nt, const double *r0,
                      const double *v0, const double *w0) {
    s->nm = nv;
    s->Xb = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    s->nb = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    s->dS = (double *)malloc(sizeof(double) * (size_t)nv);
    s->X = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    s->n = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    s->U = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    s->hl = (double *)calloc(3 * (size_t)nv, sizeof(double));
    double com[3];
    if (orc_mesh_props(verts, nv, tris, nt, s->dS, s->nb, &s->vol, com, s->Jm, &s->area) != 0) return -1;
    /* areas of the offset surface: the same triangles through Xb + OFFSET nb,
     * one third of each triangle's area to each of its vertices */
    s->dSo = (double *)calloc((size_t)nv, sizeof(double));
    for (int64_t t = 0; t < nt; ++t) {
        double P[3][3];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) P[c][a] = verts[3 * tris[3 * t + c] + a] + OFFSET * s->nb[3 * tris[3 * t + c] + a];
        double e1[3], e2[3], cr[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = P[1][a] - P[0][a];
            e2[a] = P[2][a] - P[0][a];
        }
        cross(e1, e2, cr);
        const double A = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        for (int c = 0; c < 3; ++c) s->dSo[tris[3 * t + c]] += A / 3.0;
    }
    inv3(s->Jm, s->Jminv);
    for (int64_t k = 0; k < nv; ++k)
        for (int a = 0; a < 3; ++a) s->Xb[3 * k + a] = verts[3 * k + a] - com[a];
    for (int a = 0; a < 3; ++a) {
        s->r[a] = r0[a];
        s->v[a] = v0[a];
        s->w[a] = w0[a];
        s->origin[a] = 0;
    }
    for (int i = 0; i < 9; ++i) s->d[i] = (i % 4 == 0) ? 1.0 : 0.0;
    const double m = s->p.kappa * s->vol;
    for (int a = 0; a < 3; ++a) s->L[a] = m * (s->Jm[3 * a] * w0[0] + s->Jm[3 * a + 1] * w0[1] + s->Jm[3 * a + 2] * w0[2]);
    s->has_particle = 1;
    update_markers(s);
    if (check_support(s) != 0) return -2;
    force_torque(s);
    push_history(s);
    run_ibm(s);
    return 0;
}

/* n coupled time steps in the order of Table 1.  Returns 0 or -2 if a marker
 * stencil left the window along a non-periodic axis.                        */
int orc_step(orc_sim *s, int n) {
    for (int k = 0; k < n; ++k) {
        collide_all(s);                                /* (1) collide with h_imm(t) */
        if (s->has_particle && s->p.predictor) {       /* F^, T^ for t+1 (predictor option) */
            predict(s);
            s->use_pred = 1;
        }
        if (s->has_particle) advance_particle(s);      /* (2) particle(t+1) from F(t), T(t) */
        if (s->has_particle) slide_window(s);
        if (s->has_particle) reinject(s);
        stream_all(s);                                 /* (1) stream -> f(t+1) */
        fields_from_f(s);                              /* (3) u*, sigma at t+1 */
        s->step++;
        if (!s->has_particle) continue;
        update_markers(s);
        s->use_pred = 0;
        if (check_support(s) != 0) return -2;
        force_torque(s);                               /* (3) F(t+1), T(t+1) */
        push_history(s);
        run_ibm(s);                                    /* (4) h_imm(t+1) */
    }
    return 0;
}

/* IBM cycles run so far (the paper's step: ibm_cycles - 1 per step). */
int64_t orc_ibm_cycles(const orc_sim *s) { return s->cycles; }

/* The predictor and the 6DOF update alone (tests): F, T are taken as the
 * force evaluation of the current time level (entered in the history), the
 * prediction for the next level is made, the particle advances with F, T,
 * and the motion the markers then move with is returned in vel, om. */
void orc_predictor_step(orc_sim *s, const double *F, const double *T, double *vel, double *om) {
    for (int a = 0; a < 3; ++a) {
        s->F[a] = F[a];
        s->T[a] = T[a];
    }
    push_history(s);
    predict(s);
    s->use_pred = 1;
    advance_particle(s);
    marker_motion(s, vel, om);
    s->use_pred = 0;
}

/* Particle state: r[3] (global), d[9] (rows d_i), v[3], w[3], F[3], T[3],
 * L[3], origin[3], step, vol, Jm[9], area, Fp[3]  -> 45 doubles. */
void orc_particle_state(const orc_sim *s, double *o) {
    int q = 0;
    for (int a = 0; a < 3; ++a) o[q++] = s->r[a];
    for (int a = 0; a < 9; ++a) o[q++] = s->d[a];
    for (int a = 0; a < 3; ++a) o[q++] = s->v[a];
    for (int a = 0; a < 3; ++a) o[q++] = s->w[a];
    for (int a = 0; a < 3; ++a) o[q++] = s->F[a];
    for (int a = 0; a < 3; ++a) o[q++] = s->T[a];
    for (int a = 0; a < 3; ++a) o[q++] = s->L[a];
    for (int a = 0; a < 3; ++a) o[q++] = (double)s->origin[a];
    o[q++] = (double)s->step;
    o[q++] = s->vol;
    for (int a = 0; a < 9; ++a) o[q++] = s->Jm[a];
    o[q++] = s->area;
    for (int a = 0; a < 3; ++a) o[q++] = s->Fp[a];
}

/* Marker arrays at the current time level (X, n, U: 3 per marker; dS; hl). */
void orc_markers(const orc_sim *s, double *X, double *n, double *U, double *dS, double *hl) {
    if (X) memcpy(X, s->X, sizeof(double) * 3 * (size_t)s->nm);
    if (n) memcpy(n, s->n, sizeof(double) * 3 * (size_t)s->nm);
    if (U) memcpy(U, s->U, sizeof(double) * 3 * (size_t)s->nm);
    if (dS) memcpy(dS, s->dS, sizeof(double) * (size_t)s->nm);
    if (hl) memcpy(hl, s->hl, sizeof(double) * 3 * (size_t)s->nm);
}

/* Overwrite the particle's dynamic state (tests of the 6DOF update alone). */
void orc_set_particle_dyn(orc_sim *s, const double *r, const double *d, const double *v, const double *w,
                          const double *L, const double *F, const double *T) {
    for (int a = 0; a < 3; ++a) {
        s->r[a] = r[a]; s->v[a] = v[a]; s->w[a] = w[a]; s->L[a] = L[a]; s->F[a] = F[a]; s->T[a] = T[a];
    }
    for (int a = 0; a < 9; ++a) s->d[a] = d[a];
    update_markers(s);
}

/* The 6DOF update alone with the forces held (tests). */
void orc_advance_particle_only(orc_sim *s, int n) {
    for (int k = 0; k < n; ++k) {
        advance_particle(s);
        update_markers(s);
    }
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
