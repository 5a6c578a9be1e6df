/*
 * mrs_oracle.c -- FP64 CPU oracle of the MR-STORM control cycle.
 *
 * TEST INFRASTRUCTURE ONLY (see mrs_oracle.h).  Plain loops in double
 * precision, written in the order the paper states the method:
 *   Sec. III-A (Sense / Optimize / Act, Eqs. 1-4, left-shifting),
 *   Sec. III-B (stage cost, Eq. 5),
 *   Sec. IV-A  (sphere tiling, anticipated plan, rho_b, C_dyn),
 *   Sec. IV-B  (dynamic priority alpha^(j,i)),
 *   Sec. IV-C  (Algorithm 1, the per-arm control loop).
 * No blocking, fusion or reordering beyond what those passages state.
 */
#include "mrs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_DOF 16
#define ORC_MAX_SPHERES 128

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Sampling (Sec. III-A Optimize: U_{n,h} = mu_h + eps_{n,h}, eps ~ N(0,Sigma_h)) */

/* Philox4x32 with 10 rounds, as defined by Salmon, Moraes, Dror and Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): each round
 * multiplies words 0 and 2 by two constants, forms the new words from the
 * high/low halves xor-ed with words 1, 3 and the round key, and the key is
 * bumped by two Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Top 23 bits of the word, centred in their cell: (m + 1/2) 2^-23 needs 24
 * significant bits, so it is exactly representable in float and double, and
 * it lies strictly inside (0, 1). */
double orc_uniform23(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Counter layout: word0 = sample n, word1 = step h | joint-block b << 16,
 * word2 = cycle (low 32 bits), word3 = arm | iteration << 16;
 * key = the 64-bit seed.  Each Philox call gives four words -> two
 * Box-Muller pairs -> normals for joints 4b .. 4b+3. */
void orc_normals(uint64_t seed, int arm, long long cycle, int iter, int n, int h,
                 int d, double *z)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int b = 0; 4 * b < d; ++b) {
        uint32_t ctr[4] = {(uint32_t)n, (uint32_t)h | ((uint32_t)b << 16),
                           (uint32_t)(unsigned long long)cycle,
                           (uint32_t)arm | ((uint32_t)iter << 16)};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        for (int p = 0; p < 2; ++p) {
            double u_r = orc_uniform23(x[2 * p]);
            double u_a = orc_uniform23(x[2 * p + 1]);
            double r = sqrt(-2.0 * log(u_r));
            int j0 = 4 * b + 2 * p;
            if (j0 < d) z[j0] = r * cos(two_pi * u_a);
            if (j0 + 1 < d) z[j0 + 1] = r * sin(two_pi * u_a);
        }
    }
}

/* Cholesky-Banachiewicz factor of S + jitter*I; a pivot that rounding drives
 * to or below zero is floored at 1e-12 so that the factor stays finite. */
void orc_cholesky(int d, const double *S, double jitter, double *L)
{
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = S[i * d + j] + (i == j ? jitter : 0.0);
            for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
            if (i == j) {
                L[i * d + i] = sqrt(s > 1e-12 ? s : 1e-12);
            } else {
                L[i * d + j] = s / L[j * d + j];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Kinematics (Sec. IV-A: link frames by forward kinematics, spheres at
 * constant transforms from the links).  Standard DH:
 *   T_i = T_{i-1} Rz(q_i + theta_i) Tz(d_i) Tx(a_i) Rx(alpha_i),  T_0 = base. */

static void mat4_identity(double *M)
{
    for (int i = 0; i < 16; ++i) M[i] = (i % 5 == 0) ? 1.0 : 0.0;
}

static void mat4_mul(const double *A, const double *B, double *C)
{
    double T[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[r * 4 + k] * B[k * 4 + c];
            T[r * 4 + c] = s;
        }
    memcpy(C, T, sizeof T);
}

static void rot_z(double th, double *M)
{
    mat4_identity(M);
    M[0] = cos(th); M[1] = -sin(th);
    M[4] = sin(th); M[5] = cos(th);
}

static void rot_x(double al, double *M)
{
    mat4_identity(M);
    M[5] = cos(al); M[6] = -sin(al);
    M[9] = sin(al); M[10] = cos(al);
}

static void trans(double x, double y, double z, double *M)
{
    mat4_identity(M);
    M[3] = x; M[7] = y; M[11] = z;
}

static void base_transform(const double *pose, double *M)
{
    double w = pose[3], x = pose[4], y = pose[5], z = pose[6];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    mat4_identity(M);
    M[0] = 1 - 2 * (y * y + z * z); M[1] = 2 * (x * y - w * z);     M[2] = 2 * (x * z + w * y);
    M[4] = 2 * (x * y + w * z);     M[5] = 1 - 2 * (x * x + z * z); M[6] = 2 * (y * z - w * x);
    M[8] = 2 * (x * z - w * y);     M[9] = 2 * (y * z + w * x);     M[10] = 1 - 2 * (x * x + y * y);
    M[3] = pose[0]; M[7] = pose[1]; M[11] = pose[2];
}

void orc_fk(const orc_arm *arm, const double *q, double *frames, double *spheres)
{
    double F[(ORC_MAX_DOF + 1) * 16];
    double E[16];
    base_transform(arm->base_pose, F);
    for (int i = 1; i <= arm->dof; ++i) {
        const double *p = arm->dh + 4 * (i - 1);
        double *T = F + 16 * i;
        memcpy(T, F + 16 * (i - 1), 16 * sizeof(double));
        rot_z(q[i - 1] + p[3], E); mat4_mul(T, E, T);
        trans(0, 0, p[1], E);      mat4_mul(T, E, T);
        trans(p[0], 0, 0, E);      mat4_mul(T, E, T);
        rot_x(p[2], E);            mat4_mul(T, E, T);
    }
    if (frames) memcpy(frames, F, (size_t)(arm->dof + 1) * 16 * sizeof(double));
    if (spheres) {
        for (int s = 0; s < arm->n_spheres; ++s) {
            int body = arm->sphere_body[s];
            int f = body > arm->dof ? arm->dof : body; /* tool spheres ride on frame d */
            const double *T = F + 16 * f;
            const double *pl = arm->sphere_xyzr + 4 * s;
            for (int r = 0; r < 3; ++r)
                spheres[4 * s + r] = T[4 * r] * pl[0] + T[4 * r + 1] * pl[1] +
                                     T[4 * r + 2] * pl[2] + T[4 * r + 3];
            spheres[4 * s + 3] = pl[3];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Distances.  rho_b of two spheres (Sec. IV-A) is the centre distance minus
 * both radii; a negative value is penetration depth. */

double orc_sphere_sphere(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - a[3] - b[3];
}

/* Signed distance from a sphere to an axis-aligned box (centre, half extents):
 * the exact box SDF at the sphere centre, minus the radius. */
double orc_sphere_aabb(const double *s, const double *box)
{
    double qv[3], out2 = 0.0, inside = -INFINITY;
    for (int k = 0; k < 3; ++k) {
        qv[k] = fabs(s[k] - box[k]) - box[3 + k];
        double m = qv[k] > 0.0 ? qv[k] : 0.0;
        out2 += m * m;
        if (qv[k] > inside) inside = qv[k];
    }
    if (inside > 0.0) inside = 0.0;
    return sqrt(out2) + inside - s[3];
}

/* ------------------------------------------------------------------------ */
/* Stage-cost terms (Eq. 5).  The paper names the STORM terms without their
 * formulas; the readings below are fixed once here and in the CUDA path:
 *   pose  : ||p_ee - g_p|| + w_rot * (3 - tr(R_g^T R_ee)) / 2
 *   stop  : sum_j max(0, |qd_j| - qd_max_j)^2
 *   joint : sum_j max(0, q_j - (hi_j - m))^2 + max(0, (lo_j + m) - q_j)^2
 *   world / self / dyn : the linear ramp max(0, 1 - dist / B) of Sec. IV-A. */

double orc_pose_cost(const double *T, const double *g_p, const double *g_R, double w_rot)
{
    double dx = T[3] - g_p[0], dy = T[7] - g_p[1], dz = T[11] - g_p[2];
    double tr = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) tr += g_R[3 * r + c] * T[4 * r + c];
    return sqrt(dx * dx + dy * dy + dz * dz) + w_rot * (3.0 - tr) * 0.5;
}

double orc_stop_cost(int d, const double *qd, const double *qd_max)
{
    double c = 0.0;
    for (int j = 0; j < d; ++j) {
        double e = fabs(qd[j]) - qd_max[j];
        if (e > 0.0) c += e * e;
    }
    return c;
}

double orc_joint_cost(int d, const double *q, const double *lo, const double *hi, double m)
{
    double c = 0.0;
    for (int j = 0; j < d; ++j) {
        double up = q[j] - (hi[j] - m);
        double dn = (lo[j] + m) - q[j];
        if (up > 0.0) c += up * up;
        if (dn > 0.0) c += dn * dn;
    }
    return c;
}

void orc_jacobian(const orc_arm *arm, const double *frames, double *J)
{
    const int d = arm->dof;
    const double *E = frames + 16 * d;
    for (int i = 0; i < d; ++i) {
        const double *T = frames + 16 * i;          /* frame i-1 of joint i+1 (0-based i) */
        const double z[3] = {T[2], T[6], T[10]};
        const double r[3] = {E[3] - T[3], E[7] - T[7], E[11] - T[11]};
        J[0 * d + i] = z[1] * r[2] - z[2] * r[1];
        J[1 * d + i] = z[2] * r[0] - z[0] * r[2];
        J[2 * d + i] = z[0] * r[1] - z[1] * r[0];
        J[3 * d + i] = z[0];
        J[4 * d + i] = z[1];
        J[5 * d + i] = z[2];
    }
}

/* determinant of an n x n matrix (row-major, overwritten) by Gaussian
 * elimination with partial pivoting */
static double det_inplace(int n, double *M)
{
    double det = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r * n + c]) > fabs(M[p * n + c])) p = r;
        if (M[p * n + c] == 0.0) return 0.0;
        if (p != c) {
            for (int k = 0; k < n; ++k) {
                double t = M[c * n + k];
                M[c * n + k] = M[p * n + k];
                M[p * n + k] = t;
            }
            det = -det;
        }
        det *= M[c * n + c];
        for (int r = c + 1; r < n; ++r) {
            double f = M[r * n + c] / M[c * n + c];
            for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
        }
    }
    return det;
}

double orc_manipulability(int dof, const double *J)
{
    double G[ORC_MAX_DOF * ORC_MAX_DOF];
    int n;
    if (dof >= 6) {              /* G = J J^T, 6 x 6 */
        n = 6;
        for (int a = 0; a < 6; ++a)
            for (int b = 0; b < 6; ++b) {
                double s = 0.0;
                for (int k = 0; k < dof; ++k) s += J[a * dof + k] * J[b * dof + k];
                G[a * 6 + b] = s;
            }
    } else {                     /* G = J^T J, dof x dof */
        n = dof;
        for (int a = 0; a < dof; ++a)
            for (int b = 0; b < dof; ++b) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += J[k * dof + a] * J[k * dof + b];
                G[a * dof + b] = s;
            }
    }
    double det = det_inplace(n, G);
    return det > 0.0 ? sqrt(det) : 0.0;
}

double orc_manip_cost(double w, double w0)
{
    double c = 1.0 - w / w0;
    return c > 0.0 ? c : 0.0;
}

/* C = max(0, 1 - dist/B): 0 at dist >= B, 1 at contact, linear between. */
double orc_ramp(double dist, double B)
{
    double c = 1.0 - dist / B;
    return c > 0.0 ? c : 0.0;
}

/* alpha^(j,i) = (||ee_j - g_j|| / ||ee_i - g_i||)^tau (Sec. IV-B).  Reading:
 * both distances get +1e-4 m so an arm on its goal does not divide by zero,
 * and the ratio is clamped to [1e-6, 1e6]. */
double orc_priority(double e_self, double e_other, double tau)
{
    double a = pow((e_self + 1e-4) / (e_other + 1e-4), tau);
    if (a < 1e-6) a = 1e-6;
    if (a > 1e6) a = 1e6;
    return a;
}

/* Eq. 2, written with the minimum cost subtracted (the weights are invariant
 * to a common shift of all costs; this only avoids underflow). */
void orc_weights(int K, const double *C, double lambda, double *w)
{
    double beta = C[0];
    for (int n = 1; n < K; ++n)
        if (C[n] < beta) beta = C[n];
    double Z = 0.0;
    for (int n = 0; n < K; ++n) {
        w[n] = exp(-(C[n] - beta) / lambda);
        Z += w[n];
    }
    for (int n = 0; n < K; ++n) w[n] /= Z;
}

long long orc_query_count(const orc_config *cfg, int j)
{
    long long others = 0;
    for (int i = 0; i < cfg->n_arms; ++i)
        if (i != j) others += cfg->arms[i].n_spheres;
    const orc_arm *a = &cfg->arms[j];
    return (long long)a->H * a->K * a->n_spheres * others;
}

void orc_offsets(const orc_config *cfg, int arm, long long *off_hd, long long *off_hdd,
                 long long *off_hs, long long *off_d, long long *off_k)
{
    long long hd = 0, hdd = 0, hs = 0, dd = 0, kk = 0;
    for (int a = 0; a < arm; ++a) {
        const orc_arm *A = &cfg->arms[a];
        hd += (long long)A->H * A->dof;
        hdd += (long long)A->H * A->dof * A->dof;
        hs += (long long)A->H * A->n_spheres * 4;
        dd += A->dof;
        kk += A->K;
    }
    if (off_hd) *off_hd = hd;
    if (off_hdd) *off_hdd = hdd;
    if (off_hs) *off_hs = hs;
    if (off_d) *off_d = dd;
    if (off_k) *off_k = kk;
}

void orc_init_state(const orc_config *cfg, orc_state *st)
{
    for (int a = 0; a < cfg->n_arms; ++a) {
        const orc_arm *A = &cfg->arms[a];
        long long ohd, ohdd;
        orc_offsets(cfg, a, &ohd, &ohdd, NULL, NULL, NULL);
        int d = A->dof;
        for (int h = 0; h < A->H; ++h) {
            for (int j = 0; j < d; ++j) st->mu[ohd + h * d + j] = 0.0;
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c)
                    st->Sigma[ohdd + (long long)h * d * d + r * d + c] =
                        (r == c) ? cfg->sigma_init * cfg->sigma_init : 0.0;
        }
        st->plan_valid[a] = 0;
        st->plan_stamp[a] = -1;
        st->plan_dist[a] = 0.0;
    }
    st->cycle = 0;
    st->world_t = 0.0;
}

/* A neighbour's board entry is used when it was published (Sec. IV-C: arms
 * ignore neighbours whose plans have not been published) and, with a staleness
 * limit set, is at most that many cycles old; older entries count as missing. */
static int plan_usable(const orc_config *cfg, const orc_state *st, int i)
{
    if (!st->plan_valid[i]) return 0;
    if (cfg->max_plan_age > 0 && st->cycle - st->plan_stamp[i] > cfg->max_plan_age) return 0;
    return 1;
}

static int arm_active(const orc_config *cfg, int a) { return !cfg->active || cfg->active[a]; }

/* ------------------------------------------------------------------------ */
/* Self-collision pair set of C_self (Eq. 5 names the term; the pair set is a
 * reading).  Two spheres form a pair when their bodies are at least three
 * apart along the chain (closer bodies share a joint and always touch), and
 * when their clearance at the nominal pose -- every joint at zero -- is at
 * least b_rest.  A pair that touches, or lies inside the safety band, with
 * the arm at rest belongs to the arm's build rather than to a collision; arm
 * models list such pairs as ignored, and so does this reading. */
static void rest_spheres(const orc_arm *arm, double *S_rest)
{
    double q0[ORC_MAX_DOF];
    for (int j = 0; j < arm->dof; ++j) q0[j] = 0.0;
    orc_fk(arm, q0, NULL, S_rest);
}

static int self_pair_used(const orc_arm *arm, const double *S_rest, int s1, int s2,
                          double b_rest)
{
    int gap = arm->sphere_body[s1] - arm->sphere_body[s2];
    if (gap < 0) gap = -gap;
    if (gap < 3) return 0;
    return orc_sphere_sphere(S_rest + 4 * s1, S_rest + 4 * s2) >= b_rest;
}

int orc_self_pair_used(const orc_arm *arm, int s1, int s2, double b_rest)
{
    double S_rest[ORC_MAX_SPHERES * 4];
    rest_spheres(arm, S_rest);
    return self_pair_used(arm, S_rest, s1, s2, b_rest);
}

/* ------------------------------------------------------------------------ */
/* Rollout (Sec. III-A: [C_n, X_n] = f(U_n)).  Reading of the dynamics f:
 * U are joint accelerations, integrated by semi-implicit Euler,
 *   qd_h = qd_{h-1} + U_h dt,   q_h = q_{h-1} + qd_h dt,   h = 1..H,
 * from the sensed (q, qd).  Stage h is scored on (q_h, qd_h) and the total
 * is Eq. 1 with the terminal term read as the stage cost at step H:
 *   C_n = sum_{h=1..H} gamma^{h-1} C_{n,h}. */
double orc_rollout(const orc_config *cfg, int arm, const orc_state *st, const orc_inputs *in,
                   const double *alpha_row, const double *U, double *stage,
                   double *spheres_out, double *q_out, long long *n_queries, double *sens)
{
    const orc_arm *A = &cfg->arms[arm];
    const int d = A->dof, H = A->H, NS = A->n_spheres;
    long long ohd, ohs, od;
    orc_offsets(cfg, arm, &ohd, NULL, &ohs, &od, NULL);
    double q[ORC_MAX_DOF], qd[ORC_MAX_DOF];
    double F[(ORC_MAX_DOF + 1) * 16], S[ORC_MAX_SPHERES * 4];
    for (int j = 0; j < d; ++j) {
        q[j] = in->q[od + j];
        qd[j] = in->qd[od + j];
    }
    const double *g_p = in->goal_p + 3 * arm, *g_R = in->goal_R + 9 * arm;
    double S_rest[ORC_MAX_SPHERES * 4];
    rest_spheres(A, S_rest);
    long long queries = 0;
    double total = 0.0, slope_total = 0.0;
    for (int h = 0; h < H; ++h) {
        for (int j = 0; j < d; ++j) {
            qd[j] = qd[j] + U[h * d + j] * cfg->dt;
            q[j] = q[j] + qd[j] * cfg->dt;
        }
        if (q_out)
            for (int j = 0; j < d; ++j) q_out[h * d + j] = q[j];
        orc_fk(A, q, F, S);
        if (spheres_out) memcpy(spheres_out + (size_t)h * NS * 4, S, (size_t)NS * 4 * sizeof(double));

        double c_pose = orc_pose_cost(F + 16 * d, g_p, g_R, cfg->w_rot);
        double c_stop = orc_stop_cost(d, qd, A->qd_max);
        double c_joint = orc_joint_cost(d, q, A->q_lo, A->q_hi, cfg->q_margin);
        double c_manip = 0.0;
        if (cfg->w_manip > 0.0) {
            double J[6 * ORC_MAX_DOF];
            orc_jacobian(A, F, J);
            c_manip = orc_manip_cost(orc_manipulability(d, J), cfg->manip_w0);
        }

        /* world clearance: spheres and boxes; moving spheres are predicted at
         * constant velocity to the time of step h (h+1 steps ahead). */
        double d_world = INFINITY;
        double t_h = st->world_t + (h + 1) * cfg->dt;
        for (int o = 0; o < in->n_world; ++o) {
            double ob[4];
            for (int k = 0; k < 3; ++k)
                ob[k] = in->world[4 * o + k] + (in->world_vel ? in->world_vel[3 * o + k] * t_h : 0.0);
            ob[3] = in->world[4 * o + 3];
            for (int s = 0; s < NS; ++s) {
                double dist = orc_sphere_sphere(S + 4 * s, ob);
                if (dist < d_world) d_world = dist;
            }
        }
        for (int b = 0; b < in->n_aabb; ++b)
            for (int s = 0; s < NS; ++s) {
                double dist = orc_sphere_aabb(S + 4 * s, in->aabb + 6 * b);
                if (dist < d_world) d_world = dist;
            }
        double c_coll = (in->n_world + in->n_aabb > 0) ? orc_ramp(d_world, cfg->B_world) : 0.0;

        /* self collision: the pairs of the arm's self-collision set */
        double d_self = INFINITY;
        for (int s1 = 0; s1 < NS; ++s1)
            for (int s2 = s1 + 1; s2 < NS; ++s2) {
                if (!self_pair_used(A, S_rest, s1, s2, cfg->B_self)) continue;
                double dist = orc_sphere_sphere(S + 4 * s1, S + 4 * s2);
                if (dist < d_self) d_self = dist;
            }
        double c_self = (d_self < INFINITY) ? orc_ramp(d_self, cfg->B_self) : 0.0;

        /* coordination: rho_b to every published neighbour plan at the same
         * horizon step, only up to the neighbour's own horizon */
        double c_dyn = 0.0, slope_dyn = 0.0;
        for (int i = 0; i < cfg->n_arms; ++i) {
            if (i == arm || !plan_usable(cfg, st, i)) continue;
            const orc_arm *Ai = &cfg->arms[i];
            if (h >= Ai->H) continue;
            long long ohs_i;
            orc_offsets(cfg, i, NULL, NULL, &ohs_i, NULL, NULL);
            const double *P = st->plan_spheres + ohs_i + (long long)h * Ai->n_spheres * 4;
            double rho = INFINITY;
            for (int l = 0; l < NS; ++l)
                for (int k = 0; k < Ai->n_spheres; ++k) {
                    double dist = orc_sphere_sphere(S + 4 * l, P + 4 * k);
                    if (dist < rho) rho = dist;
                    ++queries;
                }
            if (rho < 0.0) rho = 0.0;
            c_dyn += alpha_row[i] * orc_ramp(rho, cfg->B);
            if (rho > 0.0 && rho < cfg->B) slope_dyn += alpha_row[i] / cfg->B;
        }

        double c = cfg->w_pose * c_pose + cfg->w_stop * c_stop + cfg->w_joint * c_joint +
                   cfg->w_manip * c_manip + cfg->w_coll * c_coll + cfg->w_self * c_self +
                   cfg->w_dyn * c_dyn;
        if (stage) stage[h] = c;
        total += pow(cfg->gamma, (double)h) * c;
        double slope = cfg->w_pose + cfg->w_dyn * slope_dyn;
        if (d_world < cfg->B_world) slope += cfg->w_coll / cfg->B_world;
        if (d_self < cfg->B_self) slope += cfg->w_self / cfg->B_self;
        slope_total += pow(cfg->gamma, (double)h) * slope;
    }
    (void)ohd; (void)ohs;
    if (n_queries) *n_queries = queries;
    if (sens) *sens = slope_total;
    return total;
}

static int plan_usable(const orc_config *cfg, const orc_state *st, int i);
static int arm_active(const orc_config *cfg, int a);

/* ------------------------------------------------------------------------ */
/* Sense: current distance-to-goal of every arm from the measured q; priority
 * weights: own current distance against the neighbour's published one
 * (neighbours without a published plan are ignored, alpha = 0). */
static void sense_and_priority(const orc_config *cfg, const orc_state *st, const orc_inputs *in,
                               double *e_now, double *alpha)
{
    const int A = cfg->n_arms;
    for (int a = 0; a < A; ++a) {
        const orc_arm *Aa = &cfg->arms[a];
        long long od;
        orc_offsets(cfg, a, NULL, NULL, NULL, &od, NULL);
        double F[(ORC_MAX_DOF + 1) * 16];
        orc_fk(Aa, in->q + od, F, NULL);
        const double *T = F + 16 * Aa->dof;
        double dx = T[3] - in->goal_p[3 * a], dy = T[7] - in->goal_p[3 * a + 1],
               dz = T[11] - in->goal_p[3 * a + 2];
        e_now[a] = sqrt(dx * dx + dy * dy + dz * dz);
    }
    for (int a = 0; a < A; ++a)
        for (int i = 0; i < A; ++i)
            alpha[a * A + i] = (i != a && plan_usable(cfg, st, i))
                                   ? orc_priority(e_now[a], st->plan_dist[i], cfg->tau)
                                   : 0.0;
}

/* Shift (Sec. III-A) of one arm's distribution: phi_h <- phi_{h+1}; the last
 * step keeps its mean and restarts from the initial covariance. */
static void shift_arm(const orc_config *cfg, int a, double *mu, double *Sig)
{
    const orc_arm *Aa = &cfg->arms[a];
    const int d = Aa->dof, H = Aa->H;
    for (int h = 0; h + 1 < H; ++h) {
        for (int j = 0; j < d; ++j) mu[h * d + j] = mu[(h + 1) * d + j];
        for (int k = 0; k < d * d; ++k) Sig[(long long)h * d * d + k] = Sig[(long long)(h + 1) * d * d + k];
    }
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c)
            Sig[(long long)(H - 1) * d * d + r * d + c] =
                (r == c) ? cfg->sigma_init * cfg->sigma_init : 0.0;
}

/* ------------------------------------------------------------------------ */
/* One control cycle, Algorithm 1, for every arm.  All arms read the plan
 * board as it stood at the start of the cycle; the new plans are written
 * after every arm has optimised (publication at the end of the cycle). */
int orc_cycle(const orc_config *cfg, orc_state *st, const orc_inputs *in, orc_outputs *out)
{
    const int A = cfg->n_arms;
    double *e_now = (double *)calloc((size_t)A, sizeof(double));
    double *alpha = (double *)calloc((size_t)A * A, sizeof(double));
    if (!e_now || !alpha) return 1;

    sense_and_priority(cfg, st, in, e_now, alpha);

    /* Shift: not applied before the first cycle */
    if (st->cycle > 0) {
        for (int a = 0; a < A; ++a) {
            if (!arm_active(cfg, a)) continue;
            long long ohd, ohdd;
            orc_offsets(cfg, a, &ohd, &ohdd, NULL, NULL, NULL);
            shift_arm(cfg, a, st->mu + ohd, st->Sigma + ohdd);
        }
    }

    /* Optimize: K_paper iterations of SampleControls / Rollout / UpdateDistribution */
    for (int a = 0; a < A; ++a) {
        if (!arm_active(cfg, a)) continue;
        const orc_arm *Aa = &cfg->arms[a];
        const int d = Aa->dof, H = Aa->H, K = Aa->K;
        long long ohd, ohdd, od, ok;
        orc_offsets(cfg, a, &ohd, &ohdd, NULL, &od, &ok);
        double *mu = st->mu + ohd, *Sig = st->Sigma + ohdd;
        double *L = (double *)malloc(sizeof(double) * H * d * d);
        double *U = (double *)malloc(sizeof(double) * (size_t)K * H * d);
        double *C = (double *)malloc(sizeof(double) * K);
        double *w = (double *)malloc(sizeof(double) * K);
        long long *nq = (long long *)calloc((size_t)K, sizeof(long long));
        double *sn = (double *)calloc((size_t)K, sizeof(double));
        if (!L || !U || !C || !w || !nq || !sn) return 1;

        for (int it = 0; it < cfg->iterations; ++it) {
            for (int h = 0; h < H; ++h) orc_cholesky(d, Sig + h * d * d, 1e-8, L + h * d * d);

            /* SampleControls: U_{n,h} = mu_h + L_h z_{n,h} */
            for (int n = 0; n < K; ++n)
                for (int h = 0; h < H; ++h) {
                    double z[ORC_MAX_DOF];
                    orc_normals(cfg->seed, a, st->cycle, it, n, h, d, z);
                    for (int r = 0; r < d; ++r) {
                        double eps = 0.0;
                        for (int c = 0; c <= r; ++c) eps += L[h * d * d + r * d + c] * z[c];
                        U[((size_t)n * H + h) * d + r] = mu[h * d + r] + eps;
                    }
                }

            /* Rollout: every control sequence independently */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(g_threads)
#endif
            for (int n = 0; n < K; ++n)
                C[n] = orc_rollout(cfg, a, st, in, alpha + a * A, U + (size_t)n * H * d, NULL,
                                   NULL, NULL, &nq[n], &sn[n]);

            /* UpdateDistribution: Eq. 2 weights, Eq. 3 statistics, Eq. 4 EMA */
            orc_weights(K, C, cfg->lambda, w);
            for (int h = 0; h < H; ++h) {
                double mt[ORC_MAX_DOF];
                double St[ORC_MAX_DOF * ORC_MAX_DOF];
                for (int j = 0; j < d; ++j) {
                    double s = 0.0;
                    for (int n = 0; n < K; ++n) s += w[n] * U[((size_t)n * H + h) * d + j];
                    mt[j] = s;
                }
                for (int r = 0; r < d; ++r)
                    for (int c = 0; c < d; ++c) {
                        double s = 0.0;
                        for (int n = 0; n < K; ++n) {
                            const double *u = U + ((size_t)n * H + h) * d;
                            s += w[n] * (u[r] - mt[r]) * (u[c] - mt[c]);
                        }
                        St[r * d + c] = s;
                    }
                for (int j = 0; j < d; ++j)
                    mu[h * d + j] = (1.0 - cfg->alpha_mu) * mu[h * d + j] + cfg->alpha_mu * mt[j];
                for (int k = 0; k < d * d; ++k)
                    Sig[h * d * d + k] =
                        (1.0 - cfg->alpha_sigma) * Sig[h * d * d + k] + cfg->alpha_sigma * St[k];
            }

            if (it == cfg->iterations - 1) {
                /* PickBest (Sec. III-A Act): first step of the minimum-cost
                 * sequence of the final iteration; ties go to the lowest n */
                int best = 0;
                for (int n = 1; n < K; ++n)
                    if (C[n] < C[best]) best = n;
                if (out->u_star)
                    for (int j = 0; j < d; ++j) out->u_star[od + j] = U[(size_t)best * H * d + j];
                if (out->min_cost) out->min_cost[a] = C[best];
                if (out->n_star) out->n_star[a] = best;
                if (out->costs)
                    for (int n = 0; n < K; ++n) out->costs[ok + n] = C[n];
                if (out->sens)
                    for (int n = 0; n < K; ++n) out->sens[ok + n] = sn[n];
                if (out->U) {
                    long long offU = 0;
                    for (int b = 0; b < a; ++b)
                        offU += (long long)cfg->arms[b].K * cfg->arms[b].H * cfg->arms[b].dof;
                    memcpy(out->U + offU, U, sizeof(double) * (size_t)K * H * d);
                }
                if (out->n_queries) {
                    long long s = 0;
                    for (int n = 0; n < K; ++n) s += nq[n];
                    out->n_queries[a] = s;
                }
                for (int r = 0; r < out->n_dump; ++r) {
                    const int *anh = out->dump_anh + 3 * r;
                    if (anh[0] != a) continue;
                    int n = anh[1], h = anh[2];
                    double *traj = (double *)malloc(sizeof(double) * (size_t)H * Aa->n_spheres * 4);
                    double *stg = (double *)malloc(sizeof(double) * H);
                    if (!traj || !stg) return 1;
                    orc_rollout(cfg, a, st, in, alpha + a * A, U + (size_t)n * H * d, stg, traj,
                                NULL, NULL, NULL);
                    int nsmax = 0;
                    for (int b = 0; b < A; ++b)
                        if (cfg->arms[b].n_spheres > nsmax) nsmax = cfg->arms[b].n_spheres;
                    memcpy(out->dump_spheres + (size_t)r * nsmax * 4,
                           traj + (size_t)h * Aa->n_spheres * 4,
                           sizeof(double) * Aa->n_spheres * 4);
                    if (out->dump_stage) out->dump_stage[r] = stg[h];
                    free(traj);
                    free(stg);
                }
            }
        }
        free(L); free(U); free(C); free(w); free(nq); free(sn);
    }

    /* ToPlan: the mean sequence through f and forward kinematics */
    double *new_spheres = NULL, *new_q = NULL;
    {
        long long tot_hs = 0, tot_hd = 0;
        orc_offsets(cfg, A, &tot_hd, NULL, &tot_hs, NULL, NULL);
        new_spheres = (double *)malloc(sizeof(double) * (size_t)(tot_hs > 0 ? tot_hs : 1));
        new_q = (double *)malloc(sizeof(double) * (size_t)(tot_hd > 0 ? tot_hd : 1));
        if (!new_spheres || !new_q) return 1;
    }
    for (int a = 0; a < A; ++a) {
        long long ohd, ohs;
        orc_offsets(cfg, a, &ohd, NULL, &ohs, NULL, NULL);
        if (!arm_active(cfg, a)) {   /* keep what the board holds for it */
            const orc_arm *Aa = &cfg->arms[a];
            memcpy(new_spheres + ohs, st->plan_spheres + ohs,
                   sizeof(double) * Aa->H * Aa->n_spheres * 4);
            memcpy(new_q + ohd, st->plan_q + ohd, sizeof(double) * Aa->H * Aa->dof);
            continue;
        }
        orc_rollout(cfg, a, st, in, alpha + a * A, st->mu + ohd, NULL, new_spheres + ohs,
                    new_q + ohd, NULL, NULL);
    }

    /* outputs of the cycle */
    {
        long long tot_hd, tot_hdd, tot_hs, tot_d;
        orc_offsets(cfg, A, &tot_hd, &tot_hdd, &tot_hs, &tot_d, NULL);
        if (out->mean_plan) memcpy(out->mean_plan, st->mu, sizeof(double) * tot_hd);
        if (out->Sigma) memcpy(out->Sigma, st->Sigma, sizeof(double) * tot_hdd);
        if (out->plan_spheres) memcpy(out->plan_spheres, new_spheres, sizeof(double) * tot_hs);
        if (out->plan_q) memcpy(out->plan_q, new_q, sizeof(double) * tot_hd);
        if (out->dist_to_goal) memcpy(out->dist_to_goal, e_now, sizeof(double) * A);
        if (out->alpha) memcpy(out->alpha, alpha, sizeof(double) * A * A);
        /* Publish: the plan and the sensed distance-to-goal go on the board */
        memcpy(st->plan_spheres, new_spheres, sizeof(double) * tot_hs);
        memcpy(st->plan_q, new_q, sizeof(double) * tot_hd);
    }
    for (int a = 0; a < A; ++a) {
        if (!arm_active(cfg, a)) continue;
        st->plan_valid[a] = 1;
        st->plan_stamp[a] = st->cycle;
        st->plan_dist[a] = e_now[a];
    }
    st->cycle += 1;
    st->world_t += cfg->dt;
    free(new_spheres); free(new_q); free(e_now); free(alpha);
    return 0;
}

/* Costs of chosen samples of the first iteration of a cycle, one by one:
 * Sense and priority, Shift (on a copy), Cholesky, then for each requested
 * sample n its normals, U = mu + L z and the rollout.  The state is read,
 * never written.  spheres_out (may be NULL): [n_req][H][NS][4]. */
int orc_sample_costs(const orc_config *cfg, const orc_state *st, const orc_inputs *in, int arm,
                     int n_req, const int *ns, double *costs, double *spheres_out)
{
    const int A = cfg->n_arms;
    const orc_arm *Aa = &cfg->arms[arm];
    const int d = Aa->dof, H = Aa->H, NS = Aa->n_spheres;
    double *e_now = (double *)calloc((size_t)A, sizeof(double));
    double *alpha = (double *)calloc((size_t)A * A, sizeof(double));
    double *mu = (double *)malloc(sizeof(double) * H * d);
    double *Sig = (double *)malloc(sizeof(double) * H * d * d);
    double *L = (double *)malloc(sizeof(double) * H * d * d);
    double *U = (double *)malloc(sizeof(double) * H * d);
    if (!e_now || !alpha || !mu || !Sig || !L || !U) return 1;
    sense_and_priority(cfg, st, in, e_now, alpha);
    long long ohd, ohdd;
    orc_offsets(cfg, arm, &ohd, &ohdd, NULL, NULL, NULL);
    memcpy(mu, st->mu + ohd, sizeof(double) * H * d);
    memcpy(Sig, st->Sigma + ohdd, sizeof(double) * H * d * d);
    if (st->cycle > 0) shift_arm(cfg, arm, mu, Sig);
    for (int h = 0; h < H; ++h) orc_cholesky(d, Sig + h * d * d, 1e-8, L + h * d * d);
    for (int r = 0; r < n_req; ++r) {
        const int n = ns[r];
        for (int h = 0; h < H; ++h) {
            double z[ORC_MAX_DOF];
            orc_normals(cfg->seed, arm, st->cycle, 0, n, h, d, z);
            for (int i = 0; i < d; ++i) {
                double eps = 0.0;
                for (int c = 0; c <= i; ++c) eps += L[h * d * d + i * d + c] * z[c];
                U[h * d + i] = mu[h * d + i] + eps;
            }
        }
        costs[r] = orc_rollout(cfg, arm, st, in, alpha + arm * A, U, NULL,
                               spheres_out ? spheres_out + (size_t)r * H * NS * 4 : NULL, NULL, NULL,
                               NULL);
    }
    free(e_now); free(alpha); free(mu); free(Sig); free(L); free(U);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Learned clearance surrogate (not in the paper): an MLP with SiLU hidden
 * layers and a linear output, and the gradient of the mean squared error
 * against targets clipped to [-0.1, 0.3] m.  Parameter order: per hidden
 * layer W [width][in] (row-major) then b [width]; then w_out [width], b_out.
 * Input rows of in_dim values are zero-padded to in_pad. */
static double silu(double z) { return z / (1.0 + exp(-z)); }
static double dsilu(double z)
{
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

double orc_mlp_loss_grad(int in_dim, int in_pad, int width, int layers, const double *params, int n,
                         const double *x, const double *t, double *grad, double *y_out)
{
    return orc_mlp_loss_grad_w(in_dim, in_pad, width, layers, params, n, x, t, 1.0, grad, y_out);
}

double orc_mlp_loss_grad_w(int in_dim, int in_pad, int width, int layers, const double *params,
                           int n, const double *x, const double *t, double over_weight,
                           double *grad, double *y_out)
{
    const int L = layers;
    double *h = (double *)malloc(sizeof(double) * (size_t)(L + 1) * (in_pad > width ? in_pad : width));
    double *z = (double *)malloc(sizeof(double) * (size_t)L * width);
    double *dh = (double *)malloc(sizeof(double) * (in_pad > width ? in_pad : width));
    double *dz = (double *)malloc(sizeof(double) * width);
    if (!h || !z || !dh || !dz) return NAN;
    const int stride = in_pad > width ? in_pad : width;
    long long np = 0;
    for (int l = 0; l < L; ++l) np += (long long)width * (l == 0 ? in_pad : width) + width;
    np += width + 1;
    if (grad)
        for (long long i = 0; i < np; ++i) grad[i] = 0.0;
    double loss = 0.0;
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < in_pad; ++c) h[c] = c < in_dim ? x[(size_t)r * in_dim + c] : 0.0;
        long long o = 0;
        for (int l = 0; l < L; ++l) {
            const int in = l == 0 ? in_pad : width;
            const double *W = params + o, *b = params + o + (long long)width * in;
            for (int j = 0; j < width; ++j) {
                double s = b[j];
                for (int i = 0; i < in; ++i) s += W[(long long)j * in + i] * h[l * stride + i];
                z[l * width + j] = s;
                h[(l + 1) * stride + j] = silu(s);
            }
            o += (long long)width * in + width;
        }
        const double *wo = params + o, bo = params[o + width];
        double y = bo;
        for (int j = 0; j < width; ++j) y += wo[j] * h[L * stride + j];
        if (y_out) y_out[r] = y;
        double tc = t[r] < -0.1 ? -0.1 : (t[r] > 0.3 ? 0.3 : t[r]);
        double e = y - tc;
        const double we = e > 0 ? over_weight : 1.0;
        loss += we * e * e / n;
        if (!grad) continue;
        /* backward */
        double dy = 2.0 * we * e / n;
        for (int j = 0; j < width; ++j) {
            grad[o + j] += dy * h[L * stride + j];
            dh[j] = dy * wo[j];
        }
        grad[o + width] += dy;
        long long ol = o;
        for (int l = L - 1; l >= 0; --l) {
            const int in = l == 0 ? in_pad : width;
            ol -= (long long)width * in + width;
            const double *W = params + ol;
            double *gW = grad + ol, *gb = grad + ol + (long long)width * in;
            for (int j = 0; j < width; ++j) {
                dz[j] = dh[j] * dsilu(z[l * width + j]);
                gb[j] += dz[j];
                for (int i = 0; i < in; ++i) gW[(long long)j * in + i] += dz[j] * h[l * stride + i];
            }
            for (int i = 0; i < in; ++i) {
                double s = 0.0;
                for (int j = 0; j < width; ++j) s += W[(long long)j * in + i] * dz[j];
                dh[i] = s;
            }
        }
    }
    free(h); free(z); free(dh); free(dz);
    return loss;
}

void orc_pair_distance(const orc_arm *a, const orc_arm *b, int n, const double *qa,
                       const double *qb, double *out)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (int r = 0; r < n; ++r) {
        double Sa[ORC_MAX_SPHERES * 4], Sb[ORC_MAX_SPHERES * 4];
        orc_fk(a, qa + (size_t)r * a->dof, NULL, Sa);
        orc_fk(b, qb + (size_t)r * b->dof, NULL, Sb);
        double m = INFINITY;
        for (int s1 = 0; s1 < a->n_spheres; ++s1)
            for (int s2 = 0; s2 < b->n_spheres; ++s2) {
                double d = orc_sphere_sphere(Sa + 4 * s1, Sb + 4 * s2);
                if (d < m) m = d;
            }
        out[r] = m;
    }
}

/* The same clearance with arm a at the identity (its own base frame) and
 * arm b at pose_b[r] (xyz, quaternion w x y z in a's base frame), one pose
 * per row: the label of the arm-pair surrogate, whose relative poses are
 * drawn per sample. */
void orc_pair_distance_posed(const orc_arm *a, const orc_arm *b, int n, const double *qa,
                             const double *qb, const double *pose_b, double *out)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (int r = 0; r < n; ++r) {
        orc_arm A = *a, B = *b;
        const double ident[7] = {0, 0, 0, 1, 0, 0, 0};
        for (int k = 0; k < 7; ++k) {
            A.base_pose[k] = ident[k];
            B.base_pose[k] = pose_b[(size_t)r * 7 + k];
        }
        orc_pair_distance(&A, &B, 1, qa + (size_t)r * a->dof, qb + (size_t)r * b->dof, out + r);
    }
}

/* Exact self-collision clearance of joint vectors q [n][dof]: the minimum
 * over the self-collision pairs (self_pair_used, with the rest-pose band
 * b_rest = B_self) of the centre distance minus both radii (the quantity the
 * self-collision term ramps, Eq. 5); +infinity when the arm has no pair.  The
 * training label of the learned surrogate. */
void orc_self_distance(const orc_arm *arm, int n, const double *q, double b_rest, double *out)
{
    double S_rest[ORC_MAX_SPHERES * 4];
    rest_spheres(arm, S_rest);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (int r = 0; r < n; ++r) {
        double S[ORC_MAX_SPHERES * 4];
        orc_fk(arm, q + (size_t)r * arm->dof, NULL, S);
        double m = INFINITY;
        for (int s1 = 0; s1 < arm->n_spheres; ++s1)
            for (int s2 = s1 + 1; s2 < arm->n_spheres; ++s2) {
                if (!self_pair_used(arm, S_rest, s1, s2, b_rest)) continue;
                double d = orc_sphere_sphere(S + 4 * s1, S + 4 * s2);
                if (d < m) m = d;
            }
        out[r] = m;
    }
}
