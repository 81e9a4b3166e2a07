/*
 * FP64 CPU oracle for the sample-based stochastic (SBS) predictive controller
 * of Turrisi et al., "On the Benefits of GPU Sample-Based Stochastic Predictive
 * Controllers for Legged Locomotion" (IROS 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library; the two meet only
 * through seeded inputs made by the workload module.
 *
 * Everything is double precision, the quantised step frequency (Sec. IV-C)
 * included; where its FP64 value lies within rounding distance of a boundary
 * the oracle reports the margin, and the tests accept either neighbour there.
 *
 * Paper passages followed (section / equation / algorithm of the paper):
 *   sampling theta_k ~ N(theta, C), C diagonal ........ Alg. 1 (Sampling)
 *   rollout loop, cost charged on the pre-step state .. Alg. 2
 *   SRBD continuous dynamics ........................... Eq. (1), Sec. IV-A
 *   discrete dynamics x_{j+1} = f(x_j, u_j) ............ Sec. IV-A (explicit Euler)
 *   GRF spline policy Gamma = sigma(t_knot, theta_2, t)  Sec. IV-B
 *   gait: T_st = D_f / f_s, contact sequence ........... Sec. IV-C
 *   quadratic cost and step-frequency regulariser ..... Sec. V (cost equations)
 *   MPPI weights and weighted mean ..................... Sec. III-C, Alg. 5
 *   elite mean / covariance refit ...................... Alg. 1 (Update), Alg. 4
 *   Naive optimiser (best sample, covariance frozen) ... Sec. III-B, Alg. 3
 *   step frequency uniform over a discrete set, one
 *   Gaussian per frequency (Naive) ..................... Sec. V (gait optimisation), Sec. V-A
 *   world-fixed stance feet, footholds at touchdown .... Eq. (1) (p_cf,i = p_f,i - p_c), Sec. IV-D
 *   policy output constrained to the friction cone ..... Sec. IV-B
 *   one warm-started iteration per control tick ........ Sec. III-A
 *
 * Random numbers: Philox4x32-10 from Salmon, Moraes, Dror, Shaw, "Parallel
 * Random Numbers: As Easy as 1, 2, 3" (SC'11), written from that description;
 * normals by the Box-Muller transform (Box & Muller, 1958).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NX 12
#define NU 12
#define PHASE_ONE 1000000000u /* one gait cycle in units of 1e-9 cycle */
#define MAX_FREQ 8            /* largest discrete frequency set */

enum { ORC_MPPI = 0, ORC_ELITE = 1, ORC_NAIVE = 2 };
enum { ORC_OK = 0, ORC_DIVERGED = -6 };

typedef struct {
    int32_t K, H, P;         /* samples, horizon steps, spline knots (0 = one force per step) */
    int32_t method;          /* ORC_MPPI / ORC_ELITE / ORC_NAIVE */
    int32_t iterations;      /* sampling iterations per solve */
    int32_t elite_count;     /* K_e */
    int32_t adaptive;        /* 1: the step frequency is a decision variable */
    uint32_t dt_us;          /* time step in microseconds */
    uint32_t q_init;         /* nominal / initial step frequency in mHz */
    uint32_t seed, ctrl;     /* Philox key */
    double lambda;           /* MPPI temperature */
    double mass, inertia[3], foot[12], gravity[3];
    double Q[NX], R[3], w_fc, mu, rho, f_nominal;
    double f_min, f_max;
    double sigma_init, sigma_min, sigma_f_init, sigma_f_min;
    int32_t n_freq;          /* 0, or the size of a discrete step-frequency set (Naive only) */
    uint32_t freq_set[MAX_FREQ]; /* its frequencies in mHz, distinct */
    int32_t feet_mode;       /* 0: lever arms fixed in the body frame; 1: stance feet fixed on the ground */
    int32_t friction_project; /* 1: stance forces projected onto the friction cone (no penalty) */
    double w_terminal;       /* weight of the terminal state cost (0: none) */
} orc_params;

typedef struct {
    uint32_t offset[4];      /* per-leg phase offset, 1e-9 cycle */
    uint32_t duty;           /* duty factor D_f, 1e-9 cycle */
    uint32_t phase0;         /* gait phase at t = 0 of the horizon, 1e-9 cycle */
} orc_gait;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4): ten rounds of two 32x32->64  */
/* multiplies whose high halves are XORed with the other counter words and a */
/* Weyl-sequence key.                                                         */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t MUL0 = 0xD2511F53u, MUL1 = 0xCD9E8D57u;
    const uint32_t WEYL0 = 0x9E3779B9u, WEYL1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)MUL0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)MUL1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += WEYL0; k1 += WEYL1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Box-Muller on two 32-bit words.  The top 24 bits of each word give an exact
 * uniform: u1 in (0, 1], u2 in [0, 1). */
void orc_box_muller(uint32_t x, uint32_t y, double* z0, double* z1)
{
    const double two_m24 = 1.0 / 16777216.0;
    double u1 = (double)((x >> 8) + 1u) * two_m24;
    double u2 = (double)(y >> 8) * two_m24;
    double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(2.0 * M_PI * u2);
    *z1 = r * sin(2.0 * M_PI * u2);
}

/* Box-Muller on two 21-bit integers: u1 = (a + 1) 2^-21 in (0, 1] and
 * u2 = b 2^-21 in [0, 1); z0 = r cos(2 pi u2), z1 = r sin(2 pi u2) with
 * r = sqrt(-2 ln u1). */
void orc_box_muller21(uint32_t a, uint32_t b, double* z0, double* z1)
{
    const double two_m21 = 1.0 / 2097152.0;
    double u1 = (double)(a + 1u) * two_m21;
    double u2 = (double)b * two_m21;
    double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(2.0 * M_PI * u2);
    *z1 = r * sin(2.0 * M_PI * u2);
}

/* The six 21-bit integers of one 128-bit Philox block (words w0..w3): the top 21
 * bits of each word, then (low 11 bits of w0, low 10 bits of w1) and (low 11 bits
 * of w2, low 10 bits of w3), each pair joined high-to-low.  126 of the 128 bits. */
void orc_uniforms21(const uint32_t w[4], uint32_t u[6])
{
    for (int i = 0; i < 4; ++i) u[i] = w[i] >> 11;
    u[4] = ((w[0] & 0x7FFu) << 10) | (w[1] & 0x3FFu);
    u[5] = ((w[2] & 0x7FFu) << 10) | (w[3] & 0x3FFu);
}

/* The counter layout of one sample's normals.
 *   key     = (seed, controller id)
 *   counter = (sample k, draw d, iteration low word, iteration high word)
 *   draw 0  : the step-frequency normal (first Box-Muller output of the top 24
 *             bits of words 0, 1)
 *   draw d>0: force normals n = 6(d-1) .. 6(d-1)+5 from the block's six 21-bit
 *             integers: n%6 = 2p (cos) and 2p+1 (sin) from the pair (u_2p, u_2p+1).
 * Force normal n of a sample is the n-th entry of its decision vector's force
 * part (12 per step or knot), so each step uses two draws. */
double orc_normal(uint32_t seed, uint32_t ctrl, uint32_t k, uint32_t n, uint64_t iter)
{
    uint32_t ctr[4] = {k, 1u + n / 6u, (uint32_t)iter, (uint32_t)(iter >> 32)};
    uint32_t key[2] = {seed, ctrl};
    uint32_t w[4], u[6];
    orc_philox4x32_10(ctr, key, w);
    orc_uniforms21(w, u);
    unsigned slot = n % 6u, pair = slot / 2u;
    double z0, z1;
    orc_box_muller21(u[2 * pair], u[2 * pair + 1], &z0, &z1);
    return (slot % 2u == 0) ? z0 : z1;
}

/* The six force normals of draw d >= 1 (normals 6(d-1) .. 6(d-1)+5): one Philox
 * block, its six 21-bit integers and their three Box-Muller pairs, each pair
 * giving two normals.  Entry s equals orc_normal(seed, ctrl, k, 6(d-1)+s, iter). */
void orc_normals6(uint32_t seed, uint32_t ctrl, uint32_t k, uint32_t d, uint64_t iter, double out[6])
{
    uint32_t ctr[4] = {k, d, (uint32_t)iter, (uint32_t)(iter >> 32)};
    uint32_t key[2] = {seed, ctrl};
    uint32_t w[4], u[6];
    orc_philox4x32_10(ctr, key, w);
    orc_uniforms21(w, u);
    for (int p = 0; p < 3; ++p) orc_box_muller21(u[2 * p], u[2 * p + 1], &out[2 * p], &out[2 * p + 1]);
}

double orc_freq_normal(uint32_t seed, uint32_t ctrl, uint32_t k, uint64_t iter)
{
    uint32_t ctr[4] = {k, 0u, (uint32_t)iter, (uint32_t)(iter >> 32)};
    uint32_t key[2] = {seed, ctrl};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double z0, z1;
    orc_box_muller(w[0], w[1], &z0, &z1);
    return z0;
}

/* Step frequency of one sample (Sec. IV-C, frequency as decision variable theta_1):
 * f = clip(mu_f + sigma_f z, f_min, f_max), quantised to the nearest integer mHz,
 * q = floor(1000 f + 1/2), all in double precision.  *margin receives
 * |1000 f - (floor(1000 f) + 1/2)|, the distance to the nearest rounding
 * boundary: a small margin marks a sample whose rounding a lower-precision
 * evaluation of the same formula may take the other way. */
uint32_t orc_quantise_freq(double mu_f, double sigma_f, double z, double f_min, double f_max,
                           double* margin)
{
    double f = mu_f + sigma_f * z;
    if (f < f_min) f = f_min;
    if (f > f_max) f = f_max;
    double t = 1000.0 * f;
    uint32_t q = (uint32_t)floor(t + 0.5);
    if (margin) *margin = fabs((t - floor(t)) - 0.5);
    return q;
}

/* ------------------------------------------------------------------------- */
/* Gait (Sec. IV-C).  A leg's phase advances at the step frequency f_s; the   */
/* leg is in stance for the first D_f of each cycle, so T_st = D_f / f_s and  */
/* T_sw = (1 - D_f) / f_s.  Phases are integers in units of 1e-9 cycle, so the */
/* schedule is exact: at step j (time j dt) the phase advance is               */
/* j * (q mHz) * (dt_us us) = j q dt_us * 1e-9 cycle.                          */
/* ------------------------------------------------------------------------- */
int orc_stance(const orc_gait* g, int leg, uint32_t q_mhz, uint32_t dt_us, int j)
{
    uint64_t adv = (uint64_t)j * (uint64_t)q_mhz * (uint64_t)dt_us;
    uint64_t ph = ((uint64_t)g->phase0 + (uint64_t)g->offset[leg] + adv) % (uint64_t)PHASE_ONE;
    return ph < (uint64_t)g->duty ? 1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Model (Sec. IV-A, Eq. (1)).  State x = [p (world), Phi = (roll, pitch, yaw), */
/* v (world), omega (body)].  Ground reaction forces Gamma_i are world-frame, */
/* foot lever arms p_cf,i are constant in the body frame.                     */
/* ------------------------------------------------------------------------- */

/* Body-to-world rotation R = Rz(yaw) Ry(pitch) Rx(roll), row-major. */
void orc_rotation(const double rpy[3], double Rm[9])
{
    double Rx[9] = {1, 0, 0, 0, cos(rpy[0]), -sin(rpy[0]), 0, sin(rpy[0]), cos(rpy[0])};
    double Ry[9] = {cos(rpy[1]), 0, sin(rpy[1]), 0, 1, 0, -sin(rpy[1]), 0, cos(rpy[1])};
    double Rz[9] = {cos(rpy[2]), -sin(rpy[2]), 0, sin(rpy[2]), cos(rpy[2]), 0, 0, 0, 1};
    double T[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int m = 0; m < 3; ++m) s += Ry[3 * r + m] * Rx[3 * m + c];
            T[3 * r + c] = s;
        }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int m = 0; m < 3; ++m) s += Rz[3 * r + m] * T[3 * m + c];
            Rm[3 * r + c] = s;
        }
}

/* E'^{-1}(Phi): body angular velocity -> roll/pitch/yaw rates for the ZYX
 * convention above. */
void orc_euler_rates(const double rpy[3], const double w[3], double rates[3])
{
    double sr = sin(rpy[0]), cr = cos(rpy[0]);
    double tp = tan(rpy[1]), cp = cos(rpy[1]);
    rates[0] = w[0] + sr * tp * w[1] + cr * tp * w[2];
    rates[1] = cr * w[1] - sr * w[2];
    rates[2] = (sr * w[1] + cr * w[2]) / cp;
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Right-hand side of Eq. (1).  gamma: 4 legs x 3 world-frame force components,
 * already multiplied by the contact flags. f_ext: external world force (may be NULL).
 * feet: NULL for lever arms fixed in the body frame (p_cf,i = foot offset i); else
 * the world contact points (x, y) of the 4 feet on the flat ground z = 0, and
 * p_cf,i = p_f,i - p_c, so that tau_B = R^T sum_i (p_f,i - p_c) x Gamma_i. */
static void srbd_deriv(const orc_params* P, const double x[NX], const double gamma[NU],
                       const double* f_ext, const double* feet, double xdot[NX])
{
    const double* rpy = x + 3;
    const double* v = x + 6;
    const double* w = x + 9;
    double Rm[9];
    orc_rotation(rpy, Rm);
    /* translational: p_dot = v, v_dot = (1/m) sum Gamma_i + g (+ f_ext / m) */
    double F[3] = {0, 0, 0};
    for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) F[a] += gamma[3 * i + a];
    for (int a = 0; a < 3; ++a) {
        xdot[a] = v[a];
        double fe = f_ext ? f_ext[a] : 0.0;
        xdot[6 + a] = (F[a] + fe) / P->mass + P->gravity[a];
    }
    /* rotational: tau_B = sum p_cf,i x (R^T Gamma_i); omega_dot = I^{-1}(tau_B - omega x I omega) */
    double tau[3] = {0, 0, 0};
    for (int i = 0; i < 4; ++i) {
        double gb[3], r[3];
        for (int a = 0; a < 3; ++a)
            gb[a] = Rm[0 * 3 + a] * gamma[3 * i + 0] + Rm[1 * 3 + a] * gamma[3 * i + 1] +
                    Rm[2 * 3 + a] * gamma[3 * i + 2];
        if (feet) { /* body-frame lever arm R^T (p_f,i - p_c) */
            double d[3] = {feet[2 * i] - x[0], feet[2 * i + 1] - x[1], 0.0 - x[2]};
            for (int a = 0; a < 3; ++a) r[a] = Rm[0 * 3 + a] * d[0] + Rm[1 * 3 + a] * d[1] + Rm[2 * 3 + a] * d[2];
        } else {
            for (int a = 0; a < 3; ++a) r[a] = P->foot[3 * i + a];
        }
        double t[3];
        cross3(r, gb, t);
        for (int a = 0; a < 3; ++a) tau[a] += t[a];
    }
    double Iw[3] = {P->inertia[0] * w[0], P->inertia[1] * w[1], P->inertia[2] * w[2]};
    double wxIw[3];
    cross3(w, Iw, wxIw);
    for (int a = 0; a < 3; ++a) xdot[9 + a] = (tau[a] - wxIw[a]) / P->inertia[a];
    double rates[3];
    orc_euler_rates(rpy, w, rates);
    for (int a = 0; a < 3; ++a) xdot[3 + a] = rates[a];
}

void orc_srbd_deriv(const orc_params* P, const double x[NX], const double gamma[NU],
                    const double* f_ext, double xdot[NX])
{
    srbd_deriv(P, x, gamma, f_ext, NULL, xdot);
}

void orc_srbd_deriv_feet(const orc_params* P, const double x[NX], const double gamma[NU],
                         const double* f_ext, const double feet[8], double xdot[NX])
{
    srbd_deriv(P, x, gamma, f_ext, feet, xdot);
}

/* Discrete dynamics x_{j+1} = x_j + dt * f(x_j, u_j) (explicit Euler). */
static void srbd_step(const orc_params* P, const double x[NX], const double gamma[NU],
                      const double* f_ext, const double* feet, double dt, double xn[NX])
{
    double xd[NX];
    srbd_deriv(P, x, gamma, f_ext, feet, xd);
    for (int c = 0; c < NX; ++c) xn[c] = x[c] + dt * xd[c];
}

void orc_srbd_step(const orc_params* P, const double x[NX], const double gamma[NU],
                   const double* f_ext, double dt, double xn[NX])
{
    srbd_step(P, x, gamma, f_ext, NULL, dt, xn);
}

/* Foothold of leg i touching down with the body in state x (Sec. IV-D, Eq.
 * (foothold)): p_f = p_hip + (T_st / 2) v^d + sqrt(p_c,z / g) (v_c - v^d) in the
 * ground plane, with T_st = D_f / f_s the stance time of the sample's step
 * frequency (q mHz, duty in 1e-9 cycle), v^d the desired planar velocity and
 * the hip at p_c + R (foot offset x, foot offset y, 0) (the hip above the
 * nominal foot).  A CoM below the ground counts as height 0. */
void orc_foothold(const orc_params* P, const double x[NX], const double vd[2], uint32_t q_mhz, uint32_t duty,
                  int leg, double out[2])
{
    double Rm[9];
    orc_rotation(x + 3, Rm);
    double h[3] = {P->foot[3 * leg], P->foot[3 * leg + 1], 0.0};
    double Tst = ((double)duty / (double)PHASE_ONE) / (q_mhz / 1000.0);
    double s = sqrt(fmax(x[2], 0.0) / (-P->gravity[2]));
    for (int a = 0; a < 2; ++a) {
        double hw = Rm[3 * a] * h[0] + Rm[3 * a + 1] * h[1] + Rm[3 * a + 2] * h[2];
        out[a] = x[a] + hw + 0.5 * Tst * vd[a] + s * (x[6 + a] - vd[a]);
    }
}

/* Orthogonal (Euclidean) projection of a force onto the friction cone
 * {|Gamma_xy| <= mu Gamma_z} (Sec. IV-B constrains the policy output to the cone).
 * With s = |Gamma_xy| and t = Gamma_z: inside the cone nothing changes; in the
 * polar cone (mu s <= -t) the force becomes 0; otherwise it moves to the nearest
 * point of the boundary ray (mu, 1) in the (s, t) half-plane of the force,
 * lambda = (mu s + t) / (1 + mu^2), t' = lambda, s' = mu lambda. */
void orc_cone_project(double mu, const double in[3], double out[3])
{
    double s = sqrt(in[0] * in[0] + in[1] * in[1]), t = in[2];
    if (s <= mu * t) {
        out[0] = in[0]; out[1] = in[1]; out[2] = in[2];
        return;
    }
    if (mu * s <= -t) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    double lam = (mu * s + t) / (1.0 + mu * mu);
    double k = mu * lam / s;
    out[0] = k * in[0];
    out[1] = k * in[1];
    out[2] = lam;
}

/* Stage cost r(u_j, x_j, x^r_j) (Sec. V): diagonal quadratic state tracking,
 * diagonal quadratic force cost with u^r = 0, and a friction-cone penalty
 * (mu) on stance legs: max(0, |Gamma_xy| - mu Gamma_z)^2 + max(0, -Gamma_z)^2. */
double orc_stage_cost(const orc_params* P, const double x[NX], const double xr[NX],
                      const double gamma[NU], const int stance[4])
{
    double J = 0;
    for (int c = 0; c < NX; ++c) {
        double e = x[c] - xr[c];
        J += P->Q[c] * e * e;
    }
    for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) J += P->R[a] * gamma[3 * i + a] * gamma[3 * i + a];
    for (int i = 0; i < 4; ++i) {
        if (!stance[i] || P->friction_project) continue; /* projected forces need no penalty */
        double gx = gamma[3 * i], gy = gamma[3 * i + 1], gz = gamma[3 * i + 2];
        double slip = sqrt(gx * gx + gy * gy) - P->mu * gz;
        double pen = 0;
        if (slip > 0) pen += slip * slip;
        if (gz < 0) pen += gz * gz;
        J += P->w_fc * pen;
    }
    return J;
}

/* ------------------------------------------------------------------------- */
/* GRF spline (Sec. IV-B): natural cubic spline through P knots at            */
/* t_p = p T / (P - 1), T = (H - 1) dt, evaluated at t_j = j dt.  The map from */
/* knot values to samples is linear, so it is a fixed H x P basis B.           */
/* ------------------------------------------------------------------------- */
static double natural_spline_eval(int P, const double* tk, const double* y, double t)
{
    /* second derivatives M: M_0 = M_{P-1} = 0; interior rows of the standard
     * tridiagonal system, solved by the Thomas algorithm. */
    double M[64] = {0};
    if (P > 2) {
        int n = P - 2;
        double a[64], b[64], c[64], d[64];
        for (int i = 1; i <= n; ++i) {
            double h0 = tk[i] - tk[i - 1], h1 = tk[i + 1] - tk[i];
            a[i - 1] = h0;
            b[i - 1] = 2.0 * (h0 + h1);
            c[i - 1] = h1;
            d[i - 1] = 6.0 * ((y[i + 1] - y[i]) / h1 - (y[i] - y[i - 1]) / h0);
        }
        for (int i = 1; i < n; ++i) {
            double m = a[i] / b[i - 1];
            b[i] -= m * c[i - 1];
            d[i] -= m * d[i - 1];
        }
        M[n] = d[n - 1] / b[n - 1];
        for (int i = n - 1; i >= 1; --i) M[i] = (d[i - 1] - c[i - 1] * M[i + 1]) / b[i - 1];
    }
    int s = 0;
    while (s < P - 2 && t > tk[s + 1]) ++s;
    double h = tk[s + 1] - tk[s];
    double A = tk[s + 1] - t, Bt = t - tk[s];
    return M[s] * A * A * A / (6.0 * h) + M[s + 1] * Bt * Bt * Bt / (6.0 * h) +
           (y[s] / h - M[s] * h / 6.0) * A + (y[s + 1] / h - M[s + 1] * h / 6.0) * Bt;
}

void orc_knot_times(int H, int P, double dt, double* tk)
{
    double T = (H - 1) * dt;
    for (int p = 0; p < P; ++p) tk[p] = T * (double)p / (double)(P - 1);
}

/* Evaluate the spline with knot values y at an arbitrary time t in [0, T]. */
double orc_spline_at(int H, int P, double dt, const double* y, double t)
{
    double tk[64];
    orc_knot_times(H, P, dt, tk);
    return natural_spline_eval(P, tk, y, t);
}

/* B[j][p]: the spline's value at t_j when knot p is 1 and the others 0. */
void orc_spline_basis(int H, int P, double dt, double* B)
{
    double tk[64], e[64];
    orc_knot_times(H, P, dt, tk);
    for (int p = 0; p < P; ++p) {
        for (int q = 0; q < P; ++q) e[q] = (q == p) ? 1.0 : 0.0;
        for (int j = 0; j < H; ++j) B[j * P + p] = natural_spline_eval(P, tk, e, j * dt);
    }
}

/* ------------------------------------------------------------------------- */
/* Decision vector layout: a sample is theta = [force part (nf = 12 H per-step */
/* values, or 12 P knot values), step frequency (adaptive only)].  The        */
/* distribution holds one force Gaussian per frequency of a discrete set       */
/* (n_freq blocks of nf, Sec. V), else one, then the frequency entry           */
/* (adaptive only): D = n_blocks nf (+1).                                      */
/* ------------------------------------------------------------------------- */
static int nforce(const orc_params* P) { return 12 * (P->P > 0 ? P->P : P->H); }
static int nblocks(const orc_params* P) { return P->n_freq > 0 ? P->n_freq : 1; }

int orc_dim(const orc_params* P) { return nblocks(P) * nforce(P) + (P->adaptive ? 1 : 0); }

int orc_sample_dim(const orc_params* P) { return nforce(P) + (P->adaptive ? 1 : 0); }

/* Nominal step frequency (mHz) of force block b: its set value, else q_init. */
static uint32_t block_q(const orc_params* P, int b) { return P->n_freq > 0 ? P->freq_set[b] : P->q_init; }

/* Discrete step frequency (Sec. V: theta_1 takes one of a few values, drawn
 * uniformly).  The frequency draw's first Philox word gives a 24-bit uniform
 * integer u (its top bits, as in the Box-Muller uniforms); sample k takes set
 * entry floor(n u / 2^24). */
int orc_freq_bin(uint32_t seed, uint32_t ctrl, uint32_t k, uint64_t iter, int n)
{
    uint32_t ctr[4] = {k, 0u, (uint32_t)iter, (uint32_t)(iter >> 32)};
    uint32_t key[2] = {seed, ctrl}, w[4];
    orc_philox4x32_10(ctr, key, w);
    return (int)(((uint64_t)(w[0] >> 8) * (uint64_t)n) >> 24);
}

static double weight_z(const orc_params* P) { return P->mass * (-P->gravity[2]); }

/* Initial distribution (reset).  Per-step policy: at each step j every leg's mean
 * force is (0, 0, m|g| / n_j) with n_j the number of stance legs at step j of the
 * block's nominal schedule (its set frequency, else q_init), 0 when no leg is in
 * stance.  Spline policy: every knot is (0, 0, m|g| / (4 D_f)).  Variances
 * sigma_init^2; frequency mean q_init / 1000 Hz with variance sigma_f_init^2. */
static void init_step(const orc_params* P, const orc_gait* g, uint32_t q, int j, double* mu, double* var)
{
    int n = 0;
    for (int i = 0; i < 4; ++i) n += orc_stance(g, i, q, P->dt_us, j);
    double fz = n > 0 ? weight_z(P) / n : 0.0;
    for (int i = 0; i < 4; ++i) {
        mu[3 * i] = 0; mu[3 * i + 1] = 0; mu[3 * i + 2] = fz;
        for (int a = 0; a < 3; ++a) var[3 * i + a] = P->sigma_init * P->sigma_init;
    }
}

void orc_init_dist(const orc_params* P, const orc_gait* g, double* mean, double* var)
{
    int nt = P->P > 0 ? P->P : P->H, nf = nforce(P);
    for (int b = 0; b < nblocks(P); ++b) {
        double* mb = mean + (size_t)b * nf;
        double* vb = var + (size_t)b * nf;
        if (P->P > 0) {
            double fz = weight_z(P) / (4.0 * (double)g->duty / (double)PHASE_ONE);
            for (int p = 0; p < nt; ++p)
                for (int i = 0; i < 4; ++i) {
                    mb[12 * p + 3 * i] = 0; mb[12 * p + 3 * i + 1] = 0; mb[12 * p + 3 * i + 2] = fz;
                    for (int a = 0; a < 3; ++a) vb[12 * p + 3 * i + a] = P->sigma_init * P->sigma_init;
                }
        } else {
            for (int j = 0; j < nt; ++j) init_step(P, g, block_q(P, b), j, mb + 12 * j, vb + 12 * j);
        }
    }
    if (P->adaptive) {
        mean[nf] = P->q_init / 1000.0;
        var[nf] = P->sigma_f_init * P->sigma_f_init;
    }
}

/* Warm start (Sec. III-A): the previous solution, moved forward by `shift` steps
 * to the new tick.  Per-step policy: entry j takes entry j + shift; the last
 * `shift` steps are reset by the initial rule for the new gait phase.  Spline
 * policy: the new knots are the old spline evaluated at t_p + shift dt (held at
 * its end value past the horizon); variances are kept. */
void orc_warm_shift(const orc_params* P, const orc_gait* g, int shift, double* mean, double* var)
{
    if (shift <= 0) return;
    int nf = nforce(P);
    for (int b = 0; b < nblocks(P); ++b) {  /* each frequency's Gaussian moves on its own */
        double* mb = mean + (size_t)b * nf;
        double* vb = var + (size_t)b * nf;
        if (P->P > 0) {
            double dt = P->dt_us * 1e-6, T = (P->H - 1) * dt, tk[64], y[64];
            orc_knot_times(P->H, P->P, dt, tk);
            for (int c = 0; c < 12; ++c) {
                double nv[64];
                for (int p = 0; p < P->P; ++p) y[p] = mb[12 * p + c];
                for (int p = 0; p < P->P; ++p) {
                    double t = tk[p] + shift * dt;
                    if (t > T) t = T;
                    nv[p] = orc_spline_at(P->H, P->P, dt, y, t);
                }
                for (int p = 0; p < P->P; ++p) mb[12 * p + c] = nv[p];
            }
            continue;
        }
        int H = P->H;
        for (int j = 0; j < H; ++j) {
            if (j + shift < H) {
                for (int c = 0; c < 12; ++c) {
                    mb[12 * j + c] = mb[12 * (j + shift) + c];
                    vb[12 * j + c] = vb[12 * (j + shift) + c];
                }
            } else {
                init_step(P, g, block_q(P, b), j, mb + 12 * j, vb + 12 * j);
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Rollout(theta_k) (Alg. 2), for sample k of iteration `iter`:               */
/*   theta_k = mean + sd * eps_k, sd = sqrt(var) (Alg. 1 Sampling, diagonal C); */
/*         with a discrete frequency set the sample first draws its          */
/*         frequency, and                                                    */
/*         mean, var are that frequency's Gaussian (Sec. V);                 */
/*   u_j = pi(theta_k, t_j): contact flags from the sample's frequency and     */
/*         forces from the per-step values or the spline, zeroed on swing legs */
/*         (Alg. 4, function pi);                                              */
/*   J  += r(u_j, x_j, x^r_j); x_{j+1} = f(x_j, u_j).                          */
/* After the loop, an optional terminal cost w_T sum_c Q_c (x_H - x^r_{H-1})^2 */
/* (Alg. 2 leaves x_H uncosted) and, for adaptive gaits (Gaussian or discrete  */
/* frequency), rho (theta_1 - f_nominal)^2 (Sec. V).                          */
/* A non-finite cost is +inf.  q_override >= 0 replaces the sample's quantised */
/* frequency (used to evaluate both candidates of an ambiguous rounding).      */
/* ------------------------------------------------------------------------- */
typedef struct {
    const orc_params* P;
    const orc_gait* g;
    const double* x0;
    const double* xref;
    const double* f_ext;
    const double* mean;
    const double* var;
    const double* sd; /* sqrt(var), taken once per solve: C^(1/2) of the diagonal C */
    const double* B;  /* H x P spline basis, or NULL */
    uint64_t iter;
    const double* feet0; /* feet_mode 1: (x, y) of the 4 feet at t_0 */
} rollout_ctx;

/* Sign of a perturbation: a fixed integer hash of (key, a, b) mapped to +-1.
 * (Only used by the conditioning estimate below, never by the method.) */
static double pert_sign(uint64_t key, uint64_t a, uint64_t b)
{
    uint64_t z = key * 0x9E3779B97F4A7C15ull + a * 0xBF58476D1CE4E5B9ull + b * 0x94D049BB133111EBull;
    z ^= z >> 31; z *= 0xD6E8D07A4F2C6F35ull; z ^= z >> 29;
    return (z & 1ull) ? 1.0 : -1.0;
}

/* The per-solve context: the spline basis and the standard deviations are
 * formed once, not per sample. */
static rollout_ctx make_ctx(const orc_params* P, const orc_gait* g, const double* x0, const double* xref,
                            const double* f_ext, const double* feet, const double* mean, const double* var,
                            uint64_t iter)
{
    double* B = NULL;
    if (P->P > 0) {
        B = (double*)malloc(sizeof(double) * P->H * P->P);
        orc_spline_basis(P->H, P->P, P->dt_us * 1e-6, B);
    }
    int D = orc_dim(P);
    double* sd = (double*)malloc(sizeof(double) * D);
    for (int d = 0; d < D; ++d) sd[d] = sqrt(var[d]);
    rollout_ctx c = {P, g, x0, xref, f_ext, mean, var, sd, B, iter, feet};
    return c;
}

static void free_ctx(rollout_ctx* c)
{
    free((void*)c->B);
    free((void*)c->sd);
}

static double rollout_core(const rollout_ctx* c, uint32_t k, int64_t q_override, double* theta,
                           uint32_t* q_out, double* margin_out, double eps, uint64_t pkey);

static double rollout_one(const rollout_ctx* c, uint32_t k, int64_t q_override, double* theta,
                          uint32_t* q_out, double* margin_out)
{
    return rollout_core(c, k, q_override, theta, q_out, margin_out, 0.0, 0);
}

/* The rollout of Alg. 2.  With eps > 0 (conditioning estimate only) every force
 * and every state component is multiplied by (1 +- eps) after it is formed, the
 * signs fixed by pkey: a model of the per-operation rounding of a
 * lower-precision evaluation. */
static double rollout_core(const rollout_ctx* c, uint32_t k, int64_t q_override, double* theta,
                           uint32_t* q_out, double* margin_out, double eps, uint64_t pkey)
{
    const orc_params* P = c->P;
    int H = P->H, nf = nforce(P);
    double dt = P->dt_us * 1e-6;
    /* Sampling: the frequency first (it picks the force Gaussian of a discrete set) */
    uint32_t q = P->q_init;
    double margin = 1.0;
    int blk = 0;
    if (P->n_freq > 0) {
        blk = orc_freq_bin(P->seed, P->ctrl, k, c->iter, P->n_freq);
        q = P->freq_set[blk];
    }
    const double* mean = c->mean + (size_t)blk * nf;
    const double* sd = c->sd + (size_t)blk * nf;
    for (int d = 0; d < nf / 6; ++d) { /* nf is a multiple of 12: whole draws */
        double eps[6];
        orc_normals6(P->seed, P->ctrl, k, 1u + (uint32_t)d, c->iter, eps);
        for (int s = 0; s < 6; ++s) theta[6 * d + s] = mean[6 * d + s] + sd[6 * d + s] * eps[s];
    }
    if (P->adaptive) {
        double z = orc_freq_normal(P->seed, P->ctrl, k, c->iter);
        q = orc_quantise_freq(c->mean[nf], c->sd[nf], z, P->f_min, P->f_max, &margin);
    }
    if (q_override >= 0) q = (uint32_t)q_override;
    if (P->adaptive) theta[nf] = q / 1000.0;
    if (q_out) *q_out = q;
    if (margin_out) *margin_out = margin;

    double x[NX], xn[NX];
    memcpy(x, c->x0, sizeof(x));
    double feet[8];  /* world contact points (feet_mode 1) */
    int prev[4] = {1, 1, 1, 1};
    if (P->feet_mode) memcpy(feet, c->feet0, sizeof(feet));
    double J = 0;
    for (int j = 0; j < H; ++j) {
        int st[4];
        for (int i = 0; i < 4; ++i) st[i] = orc_stance(c->g, i, q, P->dt_us, j);
        if (P->feet_mode) /* a leg touching down at step j takes its foothold from x_j */
            for (int i = 0; i < 4; ++i) {
                if (st[i] && !prev[i]) orc_foothold(P, x, c->xref + NX * j + 6, q, c->g->duty, i, feet + 2 * i);
                prev[i] = st[i];
            }
        double u[NU];
        for (int n = 0; n < NU; ++n) {
            double val;
            if (P->P > 0) {
                val = 0;
                for (int p = 0; p < P->P; ++p) val += c->B[j * P->P + p] * theta[12 * p + n];
            } else {
                val = theta[12 * j + n];
            }
            u[n] = st[n / 3] ? val : 0.0;
        }
        if (P->friction_project)
            for (int i = 0; i < 4; ++i) {
                double pr[3];
                orc_cone_project(P->mu, u + 3 * i, pr);
                memcpy(u + 3 * i, pr, sizeof(pr));
            }
        if (eps > 0)
            for (int n = 0; n < NU; ++n) u[n] *= 1.0 + eps * pert_sign(pkey, 2 * (uint64_t)j, (uint64_t)n);
        J += orc_stage_cost(P, x, c->xref + NX * j, u, st);
        srbd_step(P, x, u, c->f_ext, P->feet_mode ? feet : NULL, dt, xn);
        memcpy(x, xn, sizeof(x));
        if (eps > 0)
            for (int n = 0; n < NX; ++n) x[n] *= 1.0 + eps * pert_sign(pkey, 2 * (uint64_t)j + 1, (uint64_t)n);
    }
    if (P->w_terminal > 0) { /* the state reached after the last step, against the last reference */
        double Jt = 0;
        for (int n = 0; n < NX; ++n) {
            double e = x[n] - c->xref[NX * (H - 1) + n];
            Jt += P->Q[n] * e * e;
        }
        J += P->w_terminal * Jt;
    }
    if (P->adaptive || P->n_freq > 0) {
        double d = q / 1000.0 - P->f_nominal;
        J += P->rho * d * d;
    }
    if (!isfinite(J)) J = INFINITY;
    return J;
}

/* Evaluate all K samples.  theta (K x sample dim) and margin (K) may be NULL.
 * nthreads > 1 runs samples in parallel (each sample is computed identically). */
void orc_rollout(const orc_params* P, const orc_gait* g, const double* x0, const double* xref,
                 const double* f_ext, const double* feet, const double* mean, const double* var, uint64_t iter,
                 double* J, uint32_t* q, double* theta, double* margin, int nthreads)
{
    int D = orc_sample_dim(P);
    rollout_ctx c = make_ctx(P, g, x0, xref, f_ext, feet, mean, var, iter);
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
    for (int k = 0; k < P->K; ++k) {
        double* th = theta ? theta + (size_t)k * D : (double*)malloc(sizeof(double) * D);
        uint32_t qk;
        double mk;
        J[k] = rollout_one(&c, (uint32_t)k, -1, th, &qk, &mk);
        if (q) q[k] = qk;
        if (margin) margin[k] = mk;
        if (!theta) free(th);
    }
    free_ctx(&c);
}

/* One sample with an optional forced frequency (q_override < 0: its own). */
double orc_rollout_sample(const orc_params* P, const orc_gait* g, const double* x0,
                          const double* xref, const double* f_ext, const double* feet, const double* mean,
                          const double* var, uint64_t iter, uint32_t k, int64_t q_override,
                          double* theta)
{
    rollout_ctx c = make_ctx(P, g, x0, xref, f_ext, feet, mean, var, iter);
    double J = rollout_one(&c, k, q_override, theta, NULL, NULL);
    free_ctx(&c);
    return J;
}

/* Conditioning estimate of sample k's cost (test infrastructure): the relative
 * change of J when the rollout is repeated with every force and state component
 * perturbed by a relative eps per step (four sign patterns, the largest change).
 * A cost that moves by more than the parity tolerance under rounding-sized
 * perturbations cannot be reproduced to that tolerance by any single-precision
 * evaluation; such samples are ill-conditioned. */
double orc_cost_condition(const orc_params* P, const orc_gait* g, const double* x0, const double* xref,
                          const double* f_ext, const double* feet, const double* mean, const double* var, uint64_t iter,
                          uint32_t k, double eps, double* J_out)
{
    rollout_ctx c = make_ctx(P, g, x0, xref, f_ext, feet, mean, var, iter);
    double* th = (double*)malloc(sizeof(double) * orc_dim(P));
    uint32_t q;
    double J = rollout_core(&c, k, -1, th, &q, NULL, 0.0, 0);
    double worst = 0.0;
    for (uint64_t key = 1; key <= 4; ++key) {
        double Jp = rollout_core(&c, k, (int64_t)q, th, NULL, NULL, eps, key * 1000003ull + k);
        double d;
        if (isinf(J) && isinf(Jp)) d = 0.0;
        else if (isinf(J) || isinf(Jp)) d = INFINITY;
        else d = fabs(Jp - J) / fmax(fabs(J), 1e-300);
        if (d > worst) worst = d;
    }
    if (J_out) *J_out = J;
    free(th);
    free_ctx(&c);
    return worst;
}

/* Conditioning of all K samples (parallel over samples). */
void orc_cost_condition_all(const orc_params* P, const orc_gait* g, const double* x0, const double* xref,
                            const double* f_ext, const double* feet, const double* mean, const double* var,
                            uint64_t iter, double eps, double* kappa, int nthreads)
{
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
    for (int k = 0; k < P->K; ++k)
        kappa[k] = orc_cost_condition(P, g, x0, xref, f_ext, feet, mean, var, iter, (uint32_t)k, eps, NULL);
}

/* ------------------------------------------------------------------------- */
/* MPPI UpdateMean (Sec. III-C, Alg. 5): beta = best cost,                    */
/* w~_i = exp(-(J_i - beta) / lambda), Omega = sum w~, w_i = w~_i / Omega,    */
/* theta_new = sum_i w_i theta_i.  Covariance unchanged.  Also returns the     */
/* effective sample size 1 / sum w_i^2 and beta.  Returns ORC_DIVERGED (mean   */
/* untouched) when no cost is finite.                                          */
/* ------------------------------------------------------------------------- */
int orc_mppi(const double* J, const double* theta, int K, int D, double lambda, double* mean_out,
             double* ess, double* beta_out)
{
    double beta = INFINITY;
    for (int i = 0; i < K; ++i)
        if (J[i] < beta) beta = J[i];
    if (!isfinite(beta)) return ORC_DIVERGED;
    double* w = (double*)malloc(sizeof(double) * K);
    double Omega = 0;
    for (int i = 0; i < K; ++i) {
        w[i] = isfinite(J[i]) ? exp(-(J[i] - beta) / lambda) : 0.0;
        Omega += w[i];
    }
    double s2 = 0;
    for (int i = 0; i < K; ++i) {
        w[i] /= Omega;
        s2 += w[i] * w[i];
    }
    for (int d = 0; d < D; ++d) {
        double s = 0;
        for (int i = 0; i < K; ++i) s += w[i] * theta[(size_t)i * D + d];
        mean_out[d] = s;
    }
    if (ess) *ess = 1.0 / s2;
    if (beta_out) *beta_out = beta;
    free(w);
    return ORC_OK;
}

/* Sorting (Alg. 1): order samples by (cost ascending, index ascending) and keep
 * the first K_e.  qsort over (J, k) pairs. */
typedef struct { double J; int32_t k; } cost_key;
static int cmp_cost_key(const void* a, const void* b)
{
    const cost_key* x = (const cost_key*)a;
    const cost_key* y = (const cost_key*)b;
    if (x->J < y->J) return -1;
    if (x->J > y->J) return 1;
    return (x->k > y->k) - (x->k < y->k);
}

void orc_elite_select(const double* J, int K, int Ke, int32_t* idx)
{
    cost_key* v = (cost_key*)malloc(sizeof(cost_key) * K);
    for (int i = 0; i < K; ++i) {
        v[i].J = isnan(J[i]) ? INFINITY : J[i];
        v[i].k = i;
    }
    qsort(v, K, sizeof(cost_key), cmp_cost_key);
    for (int e = 0; e < Ke; ++e) idx[e] = v[e].k;
    free(v);
}

/* Elite UpdateMean / UpdateCov (Alg. 1 Update, Alg. 4): mean and biased (maximum
 * likelihood) diagonal variance of the elite samples about the new mean, floored
 * at var_floor. */
void orc_elite_refit(const double* theta, int D, const int32_t* idx, int Ke, const double* var_floor,
                     double* mean_out, double* var_out)
{
    for (int d = 0; d < D; ++d) {
        double s = 0;
        for (int e = 0; e < Ke; ++e) s += theta[(size_t)idx[e] * D + d];
        double m = s / Ke;
        double v = 0;
        for (int e = 0; e < Ke; ++e) {
            double t = theta[(size_t)idx[e] * D + d] - m;
            v += t * t;
        }
        v /= Ke;
        if (v < var_floor[d]) v = var_floor[d];
        mean_out[d] = m;
        if (var_out) var_out[d] = v;
    }
}

/* Naive update over a discrete frequency set (Sec. III-B, Alg. 3, with one
 * Gaussian per frequency, Sec. V-A): for each set entry b, the best sample among
 * those that drew it (lowest cost, then lowest index) becomes b's force mean; an
 * entry that no finite-cost sample drew keeps its mean.  Covariances unchanged.
 * q[k] identifies sample k's entry.  best[b] gets b's winning sample or -1; the
 * return value is the entry of the best sample overall, -1 when no cost is finite. */
int orc_naive_sets(const orc_params* P, const double* J, const uint32_t* q, const double* theta,
                   double* mean, int32_t* best)
{
    int nb = P->n_freq, nf = nforce(P), Ds = orc_sample_dim(P);
    for (int b = 0; b < nb; ++b) best[b] = -1;
    for (int k = 0; k < P->K; ++k) {
        if (!isfinite(J[k])) continue;
        int b = 0;
        while (b < nb && P->freq_set[b] != q[k]) ++b;
        if (b == nb) continue; /* not a set frequency: cannot happen for this method's samples */
        if (best[b] < 0 || J[k] < J[best[b]]) best[b] = k; /* ascending k: ties keep the lower index */
    }
    int bs = -1;
    for (int b = 0; b < nb; ++b) {
        if (best[b] < 0) continue;
        if (bs < 0 || J[best[b]] < J[best[bs]] || (J[best[b]] == J[best[bs]] && best[b] < best[bs])) bs = b;
        for (int n = 0; n < nf; ++n) mean[(size_t)b * nf + n] = theta[(size_t)best[b] * Ds + n];
    }
    return bs;
}

/* First control of a distribution: the mean's forces at t_0, zeroed on legs not in
 * stance at t_0 (the contact flags at step 0 do not depend on the frequency). */
void orc_first_control(const orc_params* P, const orc_gait* g, const double* mean, double u0[NU])
{
    for (int n = 0; n < NU; ++n) {
        int st = orc_stance(g, n / 3, P->q_init, P->dt_us, 0);
        u0[n] = st ? mean[n] : 0.0; /* knot 0 of an interpolating spline is its value at t_0 */
    }
}

/* ------------------------------------------------------------------------- */
/* One solve (Alg. 4 with Alg. 1 repeated `iterations` times): warm shift,    */
/* (feet: the 4 feet's ground (x, y) at t_0 for feet_mode 1, else NULL)       */
/* then per iteration sample / evaluate / sort / update.  The distribution     */
/* (mean, var) is updated in place; iter0 is the Philox iteration counter of   */
/* the first iteration (iteration i uses iter0 + i).                           */
/* Outputs (any may be NULL): u0[12]; info[4] = {beta, ess, mean frequency,    */
/* status}; J_last, q_last (K) of the last iteration; elite_last (K_e, or the  */
/* n_freq per-frequency winners) of the last elite iteration; mppi_mean (D):   */
/* with the elite/naive method, the MPPI mean from the first iteration's       */
/* samples.  With a discrete frequency set, u0 and the mean frequency come     */
/* from the Gaussian of the best sample's frequency (the first set entry when  */
/* the last iteration has no finite cost).                                     */
/* ------------------------------------------------------------------------- */
int orc_solve(const orc_params* P, const orc_gait* g, const double* x0, const double* xref,
              const double* f_ext, const double* feet, int shift, uint64_t iter0, double* mean, double* var, double* u0,
              double* info, double* J_last, uint32_t* q_last, int32_t* elite_last,
              double* mppi_mean, int nthreads)
{
    int K = P->K, D = orc_dim(P), Ds = orc_sample_dim(P);
    orc_warm_shift(P, g, shift, mean, var);
    double* theta = (double*)malloc(sizeof(double) * (size_t)K * Ds);
    double* J = (double*)malloc(sizeof(double) * K);
    uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * K);
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (P->elite_count > 0 ? P->elite_count : 1));
    double* floor_ = (double*)malloc(sizeof(double) * D);
    for (int d = 0; d < D; ++d) floor_[d] = P->sigma_min * P->sigma_min;
    if (P->adaptive) floor_[D - 1] = P->sigma_f_min * P->sigma_f_min;
    int status = ORC_OK, bstar = 0;
    double beta = INFINITY, ess = 0;
    for (int it = 0; it < P->iterations; ++it) {
        orc_rollout(P, g, x0, xref, f_ext, feet, mean, var, iter0 + (uint64_t)it, J, q, theta, NULL, nthreads);
        double b = INFINITY;
        for (int k = 0; k < K; ++k)
            if (J[k] < b) b = J[k];
        if (!isfinite(b)) { status = ORC_DIVERGED; bstar = 0; break; }
        if (P->n_freq > 0) { /* Naive over the frequency set's Gaussians */
            int32_t best[MAX_FREQ];
            bstar = orc_naive_sets(P, J, q, theta, mean, best);
            if (elite_last) memcpy(elite_last, best, sizeof(int32_t) * P->n_freq);
            beta = b;
            ess = 1;
        } else if (P->method == ORC_MPPI) {
            orc_mppi(J, theta, K, Ds, P->lambda, mean, &ess, &beta);
        } else {
            if (it == 0 && mppi_mean) orc_mppi(J, theta, K, Ds, P->lambda, mppi_mean, NULL, NULL);
            int Ke = P->method == ORC_NAIVE ? 1 : P->elite_count;
            orc_elite_select(J, K, Ke, idx);
            if (P->method == ORC_NAIVE) {
                for (int d = 0; d < Ds; ++d) mean[d] = theta[(size_t)idx[0] * Ds + d];
            } else {
                orc_elite_refit(theta, Ds, idx, Ke, floor_, mean, var);
            }
            if (elite_last) memcpy(elite_last, idx, sizeof(int32_t) * Ke);
            beta = b;
            ess = Ke;
        }
        if (J_last) memcpy(J_last, J, sizeof(double) * K);
        if (q_last) memcpy(q_last, q, sizeof(uint32_t) * K);
    }
    if (u0) orc_first_control(P, g, mean + (size_t)bstar * nforce(P), u0);
    if (info) {
        info[0] = beta;
        info[1] = ess;
        info[2] = P->adaptive ? mean[D - 1] : block_q(P, bstar) / 1000.0;
        info[3] = status;
    }
    free(theta); free(J); free(q); free(idx); free(floor_);
    return status;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
