/*
 * mrs_oracle.h -- FP64 CPU oracle of the MR-STORM per-control-cycle MPPI update.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, no
 * header and no constant table with the CUDA path (paper_2602_10114_gb300/csrc).
 *
 * Every function follows a passage of the paper (arxiv 2602.10114, "MR-STORM:
 * Scalable Multi-Arm Control By Distributed MPC"); the citation is given as the
 * section / equation / algorithm it restates.  Where the paper is silent, the
 * reading taken is stated at the function that takes it.
 *
 * All floating point is double precision.  All arrays are caller-owned.
 */
#ifndef MRS_ORACLE_H
#define MRS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One arm's kinematic description (Sec. IV-A: spheres at constant transforms
 * from the links; standard DH chain).  Arrays are read, never written. */
typedef struct {
    int dof;            /* d, number of revolute joints (1..16) */
    int n_spheres;      /* N_S */
    int K;              /* rollouts per iteration (the paper's N) */
    int H;              /* horizon */
    const double *dh;   /* [dof][4]: a, d, alpha, theta_offset (standard DH) */
    const double *q_lo; /* [dof] joint lower limit */
    const double *q_hi; /* [dof] joint upper limit */
    const double *qd_max;       /* [dof] velocity limit of the stop cost */
    const int *sphere_body;     /* [n_spheres] body 0..dof+1 (dof+1 = tool) */
    const double *sphere_xyzr;  /* [n_spheres][4] centre in the body's frame, radius */
    double base_pose[7];        /* base position xyz + unit quaternion (w,x,y,z) */
} orc_arm;

typedef struct {
    int n_arms;
    const orc_arm *arms;
    double dt, lambda, gamma, alpha_mu, alpha_sigma, sigma_init;
    double w_pose, w_rot, w_stop, w_joint, w_coll, w_self, w_dyn;
    double B, B_world, B_self, tau;
    double q_margin;          /* soft-limit margin of the joint cost */
    int iterations;           /* optimisation iterations per cycle (paper's K) */
    uint64_t seed;            /* Philox key */
    int max_plan_age;         /* plans older than this many cycles are ignored (0: no limit) */
    const int *active;        /* [A] arms this controller optimises (NULL: all) */
    double w_manip;           /* weight of C_manip in Eq. 5 (0: term off) */
    double manip_w0;          /* manipulability below which C_manip is positive */
} orc_config;

/* Controller state carried from cycle to cycle.  Per-arm blocks are
 * concatenated in arm order (offsets: see orc_offsets). */
typedef struct {
    double *mu;            /* sum_a H_a*d_a            mean of pi_phi           */
    double *Sigma;         /* sum_a H_a*d_a*d_a        covariance of pi_phi     */
    long long cycle;       /* completed cycles (shift is skipped when 0)       */
    double world_t;        /* seconds since the world was last set             */
    /* plan board: what each arm published at the end of the previous cycle */
    int *plan_valid;       /* [A] */
    long long *plan_stamp; /* [A] cycle index at publication                   */
    double *plan_dist;     /* [A] published distance-to-goal                   */
    double *plan_spheres;  /* sum_a H_a*NS_a*4, time-major [h][k][xyzr]         */
    double *plan_q;        /* sum_a H_a*d_a joint positions of the plan        */
} orc_state;

/* Per-cycle sensed inputs (Alg. 1, Sense) and the world. */
typedef struct {
    const double *q;       /* sum_a d_a current joint positions   */
    const double *qd;      /* sum_a d_a current joint velocities  */
    const double *goal_p;  /* [A][3] goal position               */
    const double *goal_R;  /* [A][9] goal orientation, row-major  */
    int n_world;           /* world spheres */
    const double *world;   /* [n_world][4] xyz r at world_t = 0   */
    const double *world_vel; /* [n_world][3] or NULL (static)     */
    int n_aabb;
    const double *aabb;    /* [n_aabb][6] centre xyz, half extents xyz */
} orc_inputs;

/* Outputs of one cycle. */
typedef struct {
    double *mean_plan;     /* sum_a H_a*d_a   mu after the update            */
    double *Sigma;         /* sum_a H_a*d_a*d_a Sigma after the update       */
    double *plan_spheres;  /* sum_a H_a*NS_a*4 ToPlan(mu)                    */
    double *plan_q;        /* sum_a H_a*d_a                                  */
    double *u_star;        /* sum_a d_a                                      */
    double *dist_to_goal;  /* [A] */
    double *min_cost;      /* [A] min_n C_n of the last iteration           */
    int *n_star;           /* [A] argmin of the last iteration               */
    double *costs;         /* sum_a K_a  C_n of the last iteration (or NULL) */
    double *alpha;         /* [A][A] priority weights used (or NULL)        */
    long long *n_queries;  /* [A] rho_b sphere-pair evaluations (or NULL)    */
    double *sens;          /* sum_a K_a  dC_n/d(distance) of the last iteration
                              (sum of the active ramp slopes; or NULL)      */
    double *U;             /* sum_a K_a*H_a*d_a sampled U [n][h][j] of the last
                              iteration (or NULL)                            */
    /* optional sphere dumps of sampled rollouts of the last iteration */
    int n_dump;
    const int *dump_anh;   /* [n_dump][3] arm, n, h (0-based h)              */
    double *dump_spheres;  /* [n_dump][NS_max][4]                            */
    double *dump_stage;    /* [n_dump] stage cost at (n,h) (or NULL)         */
} orc_outputs;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* 23-bit uniform in (0,1) from one 32-bit word, exact in float32. */
double orc_uniform23(uint32_t x);
/* d standard normals z_{n,h,0..d-1} for (arm, cycle, iter, n, h). */
void orc_normals(uint64_t seed, int arm, long long cycle, int iter, int n, int h,
                 int d, double *z);
/* Lower Cholesky factor of S + jitter*I (row-major d x d). */
void orc_cholesky(int d, const double *S, double jitter, double *L);
/* Forward kinematics: frames [(dof+1)][16] (4x4 row-major, frame 0 = base),
 * spheres [n_spheres][4] world centre + radius. Either output may be NULL. */
void orc_fk(const orc_arm *arm, const double *q, double *frames, double *spheres);
/* Signed distances. */
double orc_sphere_sphere(const double *a, const double *b);
double orc_sphere_aabb(const double *s, const double *box);
/* Cost terms of Eq. 5 and the coordination term. */
double orc_pose_cost(const double *T_ee, const double *goal_p, const double *goal_R,
                     double w_rot);
double orc_stop_cost(int d, const double *qd, const double *qd_max);
double orc_joint_cost(int d, const double *q, const double *lo, const double *hi,
                      double margin);
double orc_ramp(double dist, double B);
double orc_priority(double e_self, double e_other, double tau);
/* MPPI weights, Eq. 2. */
void orc_weights(int K, const double *C, double lambda, double *w);
/* Number of rho_b distance queries of arm j per cycle (Sec. IV-A complexity). */
long long orc_query_count(const orc_config *cfg, int arm);

void orc_offsets(const orc_config *cfg, int arm, long long *off_hd, long long *off_hdd,
                 long long *off_hs, long long *off_d, long long *off_k);
/* Initialise state: mu = 0, Sigma = sigma^2 I, empty plan board. */
void orc_init_state(const orc_config *cfg, orc_state *st);
/* One control cycle for every arm (Alg. 1), updating st in place. */
int orc_cycle(const orc_config *cfg, orc_state *st, const orc_inputs *in,
              orc_outputs *out);
/* Rollout of one control sequence U [H][d] from (q0, qd0): stage costs
 * [H], sphere trajectory [H][NS][4] and joint trajectory [H][d] (each may
 * be NULL); n_queries (may be NULL) receives the rho_b pair count and sens
 * (may be NULL) the sensitivity of the total cost to a common error in all
 * clearance distances: sum_h gamma^h (sum of the slopes of the active ramps,
 * plus w_pose for the position error).   Used by the
 * zero-noise invariant and by ToPlan. */
double orc_rollout(const orc_config *cfg, int arm, const orc_state *st, const orc_inputs *in,
                   const double *alpha_row, const double *U, double *stage,
                   double *spheres_out, double *q_out, long long *n_queries, double *sens);
/* Costs (and optionally sphere trajectories) of chosen samples n of the
 * first iteration of the next cycle, computed one by one without running the
 * cycle; the state is not modified. */
int orc_sample_costs(const orc_config *cfg, const orc_state *st, const orc_inputs *in, int arm,
                     int n_req, const int *ns, double *costs, double *spheres_out);
/* Learned clearance surrogate (not in the paper): loss of an MLP with SiLU
 * hidden layers against clipped targets and, if grad != NULL, its gradient;
 * y_out (may be NULL) receives the outputs. */
double orc_mlp_loss_grad(int in_dim, int in_pad, int width, int layers, const double *params, int n,
                         const double *x, const double *t, double *grad, double *y_out);
/* The same with an asymmetric squared error: an over-prediction (output above
 * the clipped target: a clearance claimed larger than it is) weighs
 * over_weight, an under-prediction 1; over_weight = 1 is the plain MSE. */
double orc_mlp_loss_grad_w(int in_dim, int in_pad, int width, int layers, const double *params,
                           int n, const double *x, const double *t, double over_weight,
                           double *grad, double *y_out);
/* Self-collision pair set (reading of C_self, Eq. 5): 1 when spheres s1 and
 * s2 lie on bodies at least three apart and their clearance with every joint
 * at zero (the nominal pose) is at least b_rest (B_self in the cycle). */
int orc_self_pair_used(const orc_arm *arm, int s1, int s2, double b_rest);
/* Exact self-collision clearance of joint vectors q [n][dof] over that pair
 * set (+inf if the arm has no pair). */
void orc_self_distance(const orc_arm *arm, int n, const double *q, double b_rest, double *out);

/* Geometric Jacobian of the end-effector (the origin of frame d) in the world
 * frame, J [6][dof] row-major: for revolute joint i (axis z_{i-1} through
 * o_{i-1}, frames of orc_fk), column i = (z_{i-1} x (o_d - o_{i-1}), z_{i-1}). */
void orc_jacobian(const orc_arm *arm, const double *frames, double *J);
/* Yoshikawa manipulability, the volume of the Jacobian's velocity ellipsoid:
 * sqrt(det(J J^T)) for dof >= 6, sqrt(det(J^T J)) for dof < 6 (the product
 * of J's singular values). */
double orc_manipulability(int dof, const double *J);
/* C_manip of Eq. 5 (singularity avoidance, Sec. III-B), reading: the ramp
 * max(0, 1 - w / w0) of the manipulability w. */
double orc_manip_cost(double w, double w0);

/* Arm-to-arm clearance (the set distance of Eq. 6 without the clamp at 0):
 * for each of n rows, the minimum over all sphere pairs of arm a (at joints
 * qa [n][a->dof]) and arm b (at qb [n][b->dof]) of centre distance minus
 * radii, each arm at its own base pose.  The learned arm-pair surrogate's
 * label; negative when the arms overlap. */
void orc_pair_distance(const orc_arm *a, const orc_arm *b, int n, const double *qa,
                       const double *qb, double *out);
/* orc_pair_distance with arm a at the identity and arm b at pose_b [n][7]
 * (xyz, quaternion w x y z in a's base frame), one pose per row. */
void orc_pair_distance_posed(const orc_arm *a, const orc_arm *b, int n, const double *qa,
                             const double *qb, const double *pose_b, double *out);
void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
