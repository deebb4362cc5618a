/*
 * crowdsplat_oracle.c -- plain, slow FP64 CPU oracle for the CrowdSplat
 * crowd-synthesis path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg call it; the CUDA library never does.
 * It shares no code, header or constant table with the CUDA path.
 *
 * What it computes, in the order of CrowdSplat Sec. 2 (stage 2, crowd
 * synthesis) and of the 3D Gaussian Splatting rasteriser the paper renders
 * with (Kerbl et al. 2023, cited in Sec. 1 and Sec. 2):
 *   1. forward kinematics of each instance's 24-joint skeleton from
 *      axis-angle joint poses and a rigid root transform;
 *   2. linear blend skinning (LBS) of the shared template Gaussians: the
 *      paper animates each duplicated character by LBS (Fig. 2, Sec. 2);
 *   3. distance-based level of detail (Sec. 2: fewer Gaussians farther from
 *      the camera);
 *   4. EWA projection of each 3D Gaussian to a 2D splat, with the
 *      spherical-harmonic colour of the 3DGS rasteriser;
 *   5. the plain per-pixel definition of the image: every splat whose
 *      square support box contains the pixel centre, sorted globally by
 *      view depth, alpha-composited front to back.
 * No tiles, no sorting beyond qsort per pixel, no fusion.  Where the paper
 * is silent (it never writes the rasteriser's formulas), the 3DGS reading
 * is used: cull at view depth <= near, 2D covariance + 0.3 px^2, radius
 * ceil(3 sqrt(lambda_max)), alpha = min(0.99, o exp(q)), skip alpha < 1/255,
 * stop before transmittance drops below 1e-4.
 *
 * Parity pinned by tests/test_oracle_pins.py (closed forms, library
 * routines, invariants, brute force); no function here is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NJ 24
#define ORC_MAXL 4 /* LoD levels a subset table covers per template */

typedef struct {
    int32_t n, sh_degree;
    const float *means;       /* [n*3] metres, template local frame      */
    const float *scales;      /* [n*3] metres                            */
    const float *quats;       /* [n*4] (w,x,y,z), any norm > 0            */
    const float *opacity;     /* [n]   in [0,1]                          */
    const float *sh;          /* [n*K*3], K = (deg+1)^2, k-major per G    */
    const uint8_t *skin_idx;  /* [n*4] joint ids                         */
    const float *skin_w;      /* [n*4]                                   */
    const float *rest_joints; /* [24*3]                                  */
    const int32_t *parents;   /* [24], parents[0] = -1                   */
    const float *cov;         /* optional [n*6] xx,xy,xz,yy,yz,zz: the canonical
                                 covariance given directly (replaces
                                 scales and quats; NULL: from them)      */
} orc_template;

typedef struct {
    double R[9];  /* world -> camera rotation, row-major */
    double t[3];  /* x_cam = R x_world + t               */
    double fx, fy, cx, cy;
    int32_t width, height;
    double near_z;
} orc_camera;

typedef struct {
    int32_t n_templates;
    const orc_template *templates;
    int32_t n_instances;
    const int32_t *template_id; /* [I]      */
    const float *root;          /* [I*12]   row-major 3x4 [R|t] */
    const float *pose;          /* [I*24*3] axis-angle radians  */
    int32_t n_levels;
    const double *thresholds;   /* [L-1] ascending metres */
    const double *fractions;    /* [L]   */
    const double *scale_mult;   /* [L]   */
    int32_t skin_mode;          /* 0: LBS of means and covariances; 1: means only */
    int32_t sh_frame;           /* 0: view direction in the instance root frame; 1: world */
    orc_camera cam;
    /* optional chosen Gaussian subsets per (template t, level l), index
     * t * ORC_MAXL + l: sub_n < 0 keeps the level's prefix, otherwise the
     * level renders sub_idx[sub_off .. sub_off + sub_n) (template-local
     * indices, in that order).  sub_n may be NULL (no subsets). */
    const int32_t *sub_n;
    const int64_t *sub_off;
    const int32_t *sub_idx;
} orc_scene;

/* Windows of the boundary events (see orc_render_lattice). */
typedef struct {
    double px;        /* pixel centre within px of a support-box edge        */
    double q;         /* exponent q within q of ln(1/(255 o)) (alpha ~ 1/255) */
    double radius;    /* 3 sqrt(lambda_max) within radius of an integer       */
    double depth_rel; /* adjacent contributors with |dz| < depth_rel*max(1,z)  */
    double near_z;    /* view depth within near_z of the near plane           */
    double impact;    /* ignore events whose effect on the pixel is below this */
} orc_eps;

enum {
    ORC_EV_EDGE = 1, ORC_EV_ALPHA = 2, ORC_EV_RADIUS = 4, ORC_EV_TIE = 8,
    ORC_EV_NEAR = 16, ORC_EV_QZERO = 32, ORC_EV_LOD = 64
};

/* ------------------------------------------------------------------ */
/* small linear algebra, row-major                                      */
/* ------------------------------------------------------------------ */

static void mat3_mul(const double *A, const double *B, double *C) {
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * B[k * 3 + j];
            T[i * 3 + j] = s;
        }
    memcpy(C, T, sizeof T);
}

/* 3x4 rigid/affine composition C = A o B (both [R|t], row-major). */
static void aff_mul(const double *A, const double *B, double *C) {
    double T[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i * 4 + k] * B[k * 4 + j];
            if (j == 3) s += A[i * 4 + 3];
            T[i * 4 + j] = s;
        }
    }
    memcpy(C, T, sizeof T);
}

/* Rodrigues' formula: rotation by angle |v| about v/|v|.  Small angles use
 * the second-order series I + K + K^2/2 with K = skew(v). */
void orc_rodrigues(const double v[3], double R[9]) {
    double th = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double K[9] = {0.0, -v[2], v[1], v[2], 0.0, -v[0], -v[1], v[0], 0.0};
    double K2[9];
    mat3_mul(K, K, K2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0;
        b = 0.5;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / (th * th);
    }
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + a * K[i] + b * K2[i];
}

/* Unit quaternion (w,x,y,z) -> rotation matrix (normalised first). */
void orc_quat_to_rot(const double q_in[4], double R[9]) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------ */
/* 1. forward kinematics                                               */
/* ------------------------------------------------------------------ */

/* For one instance: local joint transforms L_j = [R_j | J_j - J_parent]
 * (L_0 = [R_0 | J_0]), global G_j = G_parent o L_j, and skinning transforms
 * B_j = Root o G_j o [I | -J_j], all 3x4 row-major.  The template's rest
 * pose has identity joint rotations, so B_j = Root when every pose is 0. */
void orc_fk(const orc_template *tp, const float *pose72, const float *root12,
            double *B_out /* [24*12] */, double *G_out /* [24*12] or NULL */) {
    double G[ORC_NJ][12];
    double root[12];
    for (int i = 0; i < 12; ++i) root[i] = root12[i];
    for (int j = 0; j < ORC_NJ; ++j) {
        double v[3] = {pose72[j * 3 + 0], pose72[j * 3 + 1], pose72[j * 3 + 2]};
        double R[9];
        orc_rodrigues(v, R);
        int p = tp->parents[j];
        double L[12];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) L[r * 4 + c] = R[r * 3 + c];
            double Jj = tp->rest_joints[j * 3 + r];
            double Jp = p >= 0 ? tp->rest_joints[p * 3 + r] : 0.0;
            L[r * 4 + 3] = Jj - Jp;
        }
        if (p < 0)
            memcpy(G[j], L, sizeof L);
        else
            aff_mul(G[p], L, G[j]);
    }
    for (int j = 0; j < ORC_NJ; ++j) {
        double unrest[12] = {1, 0, 0, -(double)tp->rest_joints[j * 3 + 0],
                             0, 1, 0, -(double)tp->rest_joints[j * 3 + 1],
                             0, 0, 1, -(double)tp->rest_joints[j * 3 + 2]};
        double tmp[12];
        aff_mul(G[j], unrest, tmp);
        aff_mul(root, tmp, B_out + j * 12);
        if (G_out) memcpy(G_out + j * 12, G[j], sizeof G[j]);
    }
}

/* ------------------------------------------------------------------ */
/* 3. distance LoD                                                      */
/* ------------------------------------------------------------------ */

static void cam_center(const orc_camera *c, double out[3]) {
    for (int i = 0; i < 3; ++i)
        out[i] = -(c->R[0 * 3 + i] * c->t[0] + c->R[1 * 3 + i] * c->t[1] + c->R[2 * 3 + i] * c->t[2]);
}

/* Band of an instance: the number of thresholds <= the distance from the
 * camera centre to the root translation (a distance equal to a threshold
 * goes to the coarser band).  Returns the level; *dist and *near_thr (the
 * distance to the closest threshold) are optional outputs. */
int orc_instance_level(const orc_scene *s, int inst, double *dist, double *near_thr) {
    double c[3];
    cam_center(&s->cam, c);
    const float *rt = s->root + (size_t)inst * 12;
    double dx = rt[3] - c[0], dy = rt[7] - c[1], dz = rt[11] - c[2];
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    int lvl = 0;
    double nt = INFINITY;
    for (int k = 0; k < s->n_levels - 1; ++k) {
        if (d >= s->thresholds[k]) lvl = k + 1;
        double e = fabs(d - s->thresholds[k]);
        if (e < nt) nt = e;
    }
    if (dist) *dist = d;
    if (near_thr) *near_thr = nt;
    return lvl;
}

/* Number of Gaussians in level `lvl` of a template of n: f * n rounded
 * half up, clamped to [0, n] (the level keeps the first N_l Gaussians). */
int orc_level_count(const orc_scene *s, int lvl, int n) {
    double c = floor(s->fractions[lvl] * (double)n + 0.5);
    if (c < 0.0) c = 0.0;
    if (c > n) c = n;
    return (int)c;
}

/* Size of level `lvl` of template t: its chosen subset's length, else the
 * prefix of orc_level_count. */
int orc_level_size(const orc_scene *s, int t, int lvl) {
    if (s->sub_n && s->sub_n[t * ORC_MAXL + lvl] >= 0) return s->sub_n[t * ORC_MAXL + lvl];
    return orc_level_count(s, lvl, s->templates[t].n);
}

/* Template-local index of the k-th Gaussian of level `lvl` of template t. */
int orc_level_gauss(const orc_scene *s, int t, int lvl, int k) {
    if (s->sub_n && s->sub_n[t * ORC_MAXL + lvl] >= 0) return s->sub_idx[s->sub_off[t * ORC_MAXL + lvl] + k];
    return k;
}

/* ------------------------------------------------------------------ */
/* 4. spherical harmonics (real basis, 3DGS sign convention)            */
/* ------------------------------------------------------------------ */

/* Real SH basis up to degree 3 at unit direction (x,y,z), order m = -l..l
 * within each degree.  The convention is that of the 3DGS rasteriser:
 * degree 1 = C1 (-y, z, -x).  Constants from their closed forms. */
void orc_sh_basis(int deg, const double d[3], double *Y /* [(deg+1)^2] */) {
    const double x = d[0], y = d[1], z = d[2];
    const double PI = 3.14159265358979323846;
    Y[0] = 0.5 / sqrt(PI);
    if (deg < 1) return;
    double c1 = sqrt(3.0 / (4.0 * PI));
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (deg < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    double a = 0.5 * sqrt(15.0 / PI), b = 0.25 * sqrt(5.0 / PI), e = 0.25 * sqrt(15.0 / PI);
    Y[4] = a * x * y;
    Y[5] = -a * y * z;
    Y[6] = b * (2.0 * zz - xx - yy);
    Y[7] = -a * x * z;
    Y[8] = e * (xx - yy);
    if (deg < 3) return;
    double k0 = 0.25 * sqrt(35.0 / (2.0 * PI));
    double k1 = 0.5 * sqrt(105.0 / PI);
    double k2 = 0.25 * sqrt(21.0 / (2.0 * PI));
    double k3 = 0.25 * sqrt(7.0 / PI);
    double k5 = 0.25 * sqrt(105.0 / PI);
    Y[9] = -k0 * y * (3.0 * xx - yy);
    Y[10] = k1 * x * y * z;
    Y[11] = -k2 * y * (4.0 * zz - xx - yy);
    Y[12] = k3 * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -k2 * x * (4.0 * zz - xx - yy);
    Y[14] = k5 * z * (xx - yy);
    Y[15] = -k0 * x * (xx - 3.0 * yy);
}

/* ------------------------------------------------------------------ */
/* 2 + 4. one Gaussian of one instance: LBS, projection, colour         */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t valid;      /* survived every cull                                  */
    int32_t boxed;      /* projected with a positive 2D covariance               */
    int32_t on_image;   /* support box contains a pixel centre of the image      */
    int32_t r;          /* support half-width in pixels                         */
    double mu[3];       /* posed mean, world                                    */
    double cov3[6];     /* posed covariance, world (xx,xy,xz,yy,yz,zz)          */
    double tcam[3];     /* mean in camera space                                 */
    double cov2[3];     /* 2D covariance incl. +0.3 (a, b, c)                    */
    double conic[3];    /* inverse 2D covariance (A, B, C)                       */
    double u, v;        /* projected mean, pixels                               */
    double depth;       /* tcam[2]                                              */
    double r_exact;     /* 3 sqrt(lambda_max) before rounding up                */
    double opacity;
    double rgb[3];
} orc_splat;

/* Everything for Gaussian g of instance `inst` at LoD level `lvl`, given the
 * instance's skinning transforms B (from orc_fk). */
void orc_splat_compute(const orc_scene *s, int inst, const double *B, int lvl, int g,
                       orc_splat *o) {
    const orc_template *tp = &s->templates[s->template_id[inst]];
    const orc_camera *cam = &s->cam;
    memset(o, 0, sizeof *o);
    /* LBS: M = sum_k w_k B_{idx_k}; mu' = M [mu; 1]; Sigma' = A Sigma A^T */
    double M[12] = {0};
    for (int k = 0; k < 4; ++k) {
        double w = tp->skin_w[(size_t)g * 4 + k];
        int j = tp->skin_idx[(size_t)g * 4 + k];
        for (int e = 0; e < 12; ++e) M[e] += w * B[j * 12 + e];
    }
    double mu[3] = {tp->means[(size_t)g * 3 + 0], tp->means[(size_t)g * 3 + 1], tp->means[(size_t)g * 3 + 2]};
    for (int r = 0; r < 3; ++r)
        o->mu[r] = M[r * 4 + 0] * mu[0] + M[r * 4 + 1] * mu[1] + M[r * 4 + 2] * mu[2] + M[r * 4 + 3];
    /* canonical covariance Sigma = R(q) S S^T R(q)^T, S = diag(m_l * s),
     * or m_l^2 times the covariance given directly */
    double m = s->scale_mult[lvl];
    double Sig[9];
    if (tp->cov) {
        const float *c = tp->cov + (size_t)g * 6;
        const double m2 = m * m;
        Sig[0] = m2 * c[0]; Sig[1] = m2 * c[1]; Sig[2] = m2 * c[2];
        Sig[3] = m2 * c[1]; Sig[4] = m2 * c[3]; Sig[5] = m2 * c[4];
        Sig[6] = m2 * c[2]; Sig[7] = m2 * c[4]; Sig[8] = m2 * c[5];
    } else {
        double q[4] = {tp->quats[(size_t)g * 4 + 0], tp->quats[(size_t)g * 4 + 1],
                       tp->quats[(size_t)g * 4 + 2], tp->quats[(size_t)g * 4 + 3]};
        double Rq[9];
        orc_quat_to_rot(q, Rq);
        double S[3] = {m * tp->scales[(size_t)g * 3 + 0], m * tp->scales[(size_t)g * 3 + 1],
                       m * tp->scales[(size_t)g * 3 + 2]};
        double RS[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) RS[i * 3 + j] = Rq[i * 3 + j] * S[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += RS[i * 3 + k] * RS[j * 3 + k];
                Sig[i * 3 + j] = acc;
            }
    }
    double Sp[9];
    if (s->skin_mode == 0) {
        /* Sigma' = A Sigma A^T with A the 3x3 part of M */
        double A[9] = {M[0], M[1], M[2], M[4], M[5], M[6], M[8], M[9], M[10]};
        double AS[9];
        mat3_mul(A, Sig, AS);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += AS[i * 3 + k] * A[j * 3 + k];
                Sp[i * 3 + j] = acc;
            }
    } else {
        /* means only: the covariance follows the root rotation alone */
        const float *rt = s->root + (size_t)inst * 12;
        double A[9] = {rt[0], rt[1], rt[2], rt[4], rt[5], rt[6], rt[8], rt[9], rt[10]};
        double AS[9];
        mat3_mul(A, Sig, AS);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += AS[i * 3 + k] * A[j * 3 + k];
                Sp[i * 3 + j] = acc;
            }
    }
    o->cov3[0] = Sp[0]; o->cov3[1] = Sp[1]; o->cov3[2] = Sp[2];
    o->cov3[3] = Sp[4]; o->cov3[4] = Sp[5]; o->cov3[5] = Sp[8];
    o->opacity = tp->opacity[g];

    /* view transform */
    for (int r = 0; r < 3; ++r)
        o->tcam[r] = cam->R[r * 3 + 0] * o->mu[0] + cam->R[r * 3 + 1] * o->mu[1] +
                     cam->R[r * 3 + 2] * o->mu[2] + cam->t[r];
    double tx = o->tcam[0], ty = o->tcam[1], tz = o->tcam[2];
    o->depth = tz;
    /* near-plane cull (view depth <= near); the projection below is still
     * evaluated for depths just behind the plane so that the compositing
     * can flag splats an FP32 evaluation might keep */
    int near_culled = tz <= cam->near_z;
    if (tz <= 1e-6) return;

    /* EWA: Sigma2D = J W Sigma' W^T J^T + 0.3 I, J evaluated at the mean
     * with x/z, y/z clamped to 1.3x the half field of view */
    double limx = 1.3 * (0.5 * cam->width) / cam->fx;
    double limy = 1.3 * (0.5 * cam->height) / cam->fy;
    double txz = tx / tz, tyz = ty / tz;
    if (txz < -limx) txz = -limx;
    if (txz > limx) txz = limx;
    if (tyz < -limy) tyz = -limy;
    if (tyz > limy) tyz = limy;
    double J[6] = {cam->fx / tz, 0.0, -cam->fx * txz / tz, 0.0, cam->fy / tz, -cam->fy * tyz / tz};
    double Vc[9]; /* W Sigma' W^T */
    {
        double WS[9];
        mat3_mul(cam->R, Sp, WS);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += WS[i * 3 + k] * cam->R[j * 3 + k];
                Vc[i * 3 + j] = acc;
            }
    }
    double JV[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += J[i * 3 + k] * Vc[k * 3 + j];
            JV[i * 3 + j] = acc;
        }
    double c2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += JV[i * 3 + k] * J[j * 3 + k];
            c2[i * 2 + j] = acc;
        }
    double a = c2[0] + 0.3, b = c2[1], c = c2[3] + 0.3;
    o->cov2[0] = a; o->cov2[1] = b; o->cov2[2] = c;
    double det = a * c - b * b;
    if (det <= 0.0) return;
    o->conic[0] = c / det;
    o->conic[1] = -b / det;
    o->conic[2] = a / det;
    double mid = 0.5 * (a + c);
    double disc = mid * mid - det;
    if (disc < 0.1) disc = 0.1;
    double lam = mid + sqrt(disc);
    o->r_exact = 3.0 * sqrt(lam);
    o->r = (int32_t)ceil(o->r_exact);
    o->u = cam->fx * tx / tz + cam->cx;
    o->v = cam->fy * ty / tz + cam->cy;
    if (o->r <= 0) return;
    o->boxed = 1;
    /* support box must contain at least one pixel centre of the image */
    double i0 = ceil(o->u - o->r - 0.5), i1 = floor(o->u + o->r - 0.5);
    double j0 = ceil(o->v - o->r - 0.5), j1 = floor(o->v + o->r - 0.5);
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    if (i1 > cam->width - 1) i1 = cam->width - 1;
    if (j1 > cam->height - 1) j1 = cam->height - 1;
    if (i0 > i1 || j0 > j1) return;
    o->on_image = 1;

    /* colour: SH at the viewing direction (camera centre -> mean), in the
     * instance root frame (sh_frame 0) or the world frame (1) */
    double cc[3];
    cam_center(cam, cc);
    double d[3] = {o->mu[0] - cc[0], o->mu[1] - cc[1], o->mu[2] - cc[2]};
    if (s->sh_frame == 0) {
        const float *rt = s->root + (size_t)inst * 12;
        double dl[3];
        for (int i = 0; i < 3; ++i) dl[i] = rt[0 * 4 + i] * d[0] + rt[1 * 4 + i] * d[1] + rt[2 * 4 + i] * d[2];
        memcpy(d, dl, sizeof dl);
    }
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= dn; d[1] /= dn; d[2] /= dn;
    int deg = tp->sh_degree;
    int K = (deg + 1) * (deg + 1);
    double Y[16];
    orc_sh_basis(deg, d, Y);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += Y[k] * tp->sh[((size_t)g * K + k) * 3 + ch];
        acc += 0.5;
        o->rgb[ch] = acc < 0.0 ? 0.0 : acc;
    }
    o->valid = !near_culled;
}

/* Per-instance splats for parity checks: all Gaussians of the instance's
 * LoD level, in level order (the prefix, or the chosen subset's order).
 * Arrays have `count` rows (count = level size, returned).  Any output
 * pointer may be NULL. */
int orc_project_instance(const orc_scene *s, int inst, int32_t *level_out,
                         int32_t *valid, int32_t *radius, double *uv /*[n*2]*/,
                         double *conic /*[n*3]*/, double *depth, double *rgb /*[n*3]*/,
                         double *opacity, double *mu /*[n*3]*/, double *cov3 /*[n*6]*/,
                         double *cov2 /*[n*3]*/, double *r_exact, double *B_out /*[24*12]*/) {
    const orc_template *tp = &s->templates[s->template_id[inst]];
    double B[ORC_NJ * 12];
    orc_fk(tp, s->pose + (size_t)inst * 72, s->root + (size_t)inst * 12, B, NULL);
    if (B_out) memcpy(B_out, B, sizeof B);
    int lvl = orc_instance_level(s, inst, NULL, NULL);
    if (level_out) *level_out = lvl;
    const int t = s->template_id[inst];
    int n = orc_level_size(s, t, lvl);
    #pragma omp parallel for schedule(static)
    for (int g = 0; g < n; ++g) {
        orc_splat sp;
        orc_splat_compute(s, inst, B, lvl, orc_level_gauss(s, t, lvl, g), &sp);
        if (valid) valid[g] = sp.valid;
        if (radius) radius[g] = sp.r;
        if (uv) { uv[g * 2] = sp.u; uv[g * 2 + 1] = sp.v; }
        if (conic) for (int i = 0; i < 3; ++i) conic[g * 3 + i] = sp.conic[i];
        if (depth) depth[g] = sp.depth;
        if (rgb) for (int i = 0; i < 3; ++i) rgb[g * 3 + i] = sp.rgb[i];
        if (opacity) opacity[g] = sp.opacity;
        if (mu) for (int i = 0; i < 3; ++i) mu[g * 3 + i] = sp.mu[i];
        if (cov3) for (int i = 0; i < 6; ++i) cov3[g * 6 + i] = sp.cov3[i];
        if (cov2) for (int i = 0; i < 3; ++i) cov2[g * 3 + i] = sp.cov2[i];
        if (r_exact) r_exact[g] = sp.r_exact;
    }
    return n;
}

/* ------------------------------------------------------------------ */
/* 5. per-pixel compositing over a lattice of pixels                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t pix;      /* lattice index                          */
    int32_t inst, g;  /* g: position in the instance's level     */
    int64_t gt;       /* Gaussian's index over all templates     */
    int32_t r;
    int32_t near_ev;  /* view depth close to the near plane      */
    int32_t rad_ev;   /* radius close to an integer              */
    int32_t valid;    /* composited (not culled by the near plane) */
    double depth, u, v, A, B, C, o, rgb[3];
} orc_entry;

typedef struct {
    orc_entry *e;
    size_t n, cap;
} orc_vec;

static void vec_push(orc_vec *v, const orc_entry *e) {
    if (v->n == v->cap) {
        size_t nc = v->cap ? v->cap * 2 : 1024;
        orc_entry *ne = (orc_entry *)realloc(v->e, nc * sizeof(orc_entry));
        if (!ne) abort();
        v->e = ne;
        v->cap = nc;
    }
    v->e[v->n++] = *e;
}

static int cmp_entry(const void *pa, const void *pb) {
    const orc_entry *a = (const orc_entry *)pa, *b = (const orc_entry *)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    if (a->inst != b->inst) return a->inst < b->inst ? -1 : 1;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return 0;
}

static double dmax(double a, double b) { return a > b ? a : b; }

/* Render the pixels (ox + i*sx, oy + j*sy), i < nx, j < ny.
 *
 * Each pixel's colour is the front-to-back composite, over every splat
 * whose support box |p - (u,v)|_inf <= r contains the pixel centre p,
 * ordered by (view depth, instance, Gaussian):
 *   q = -(A dx^2 + C dy^2)/2 - B dx dy;  skip q > 0;
 *   alpha = min(0.99, o e^q);  skip alpha < 1/255;
 *   T' = T (1 - alpha);  stop (without this splat) if T' < 1e-4;
 *   C += c alpha T;  T = T'.
 * Outputs RGB = C (black background), A = 1 - T, wsum = sum alpha T, and
 * (optional) contrib[gt] += alpha T for each composited Gaussian, gt its
 * index over all templates (template t's Gaussians follow those of
 * templates 0 .. t-1).
 *
 * Boundary events: where an FP32 evaluation of the same definition may take
 * the other branch of a discontinuous decision, the pixel is flagged if
 * that branch can move the pixel by more than eps->impact (an upper bound
 * of the jump: 2 alpha T max(1, |c|)).  Event kinds (flags bitmask): box
 * edge within eps->px of the centre; alpha within eps->q (in exponent) of
 * 1/255; radius within eps->radius of an integer (pixel in the outer ring);
 * adjacent contributors closer in depth than eps->depth_rel; view depth
 * within eps->near_z of the near plane; q within 1e-6 of 0; instance
 * distance within 1e-4 m of an LoD threshold.
 * Returns 0, or -1 on allocation failure. */
int orc_render_lattice(const orc_scene *s, const orc_eps *eps, int ox, int oy, int sx, int sy,
                       int nx, int ny, double *rgba /*[ny*nx*4]*/, double *wsum /*[ny*nx]*/,
                       uint32_t *flags /*[ny*nx]*/, double *impact /*[ny*nx]*/,
                       int32_t *ncontrib /*[ny*nx]*/, double *contrib /*[total Gaussians] or NULL*/) {
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    orc_vec *vecs = (orc_vec *)calloc((size_t)nthreads, sizeof(orc_vec));
    uint8_t *lod_ev = (uint8_t *)calloc((size_t)(s->n_instances > 0 ? s->n_instances : 1), 1);
    int64_t *g_off = (int64_t *)calloc((size_t)s->n_templates + 1, sizeof(int64_t));
    if (!vecs || !lod_ev || !g_off) return -1;
    for (int t = 0; t < s->n_templates; ++t) g_off[t + 1] = g_off[t] + s->templates[t].n;
    const double margin_px = eps->px;

    #pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        orc_vec *vec = &vecs[tid];
        #pragma omp for schedule(dynamic, 1)
        for (int inst = 0; inst < s->n_instances; ++inst) {
            const orc_template *tp = &s->templates[s->template_id[inst]];
            double B[ORC_NJ * 12];
            orc_fk(tp, s->pose + (size_t)inst * 72, s->root + (size_t)inst * 12, B, NULL);
            double nt;
            int lvl = orc_instance_level(s, inst, NULL, &nt);
            if (nt < 1e-4) lod_ev[inst] = 1;
            const int t = s->template_id[inst];
            int n = orc_level_size(s, t, lvl);
            for (int g = 0; g < n; ++g) {
                orc_splat sp;
                const int gl = orc_level_gauss(s, t, lvl, g);
                orc_splat_compute(s, inst, B, lvl, gl, &sp);
                int near_ev = fabs(sp.depth - s->cam.near_z) < eps->near_z;
                /* keep contributors, and near-plane culls close to the plane */
                if (!sp.on_image || (!sp.valid && !near_ev)) continue;
                int rad_ev = fabs(sp.r_exact - floor(sp.r_exact + 0.5)) < eps->radius;
                double ext = (double)sp.r + margin_px + (rad_ev ? 1.0 : 0.0);
                /* lattice pixels with centre in [u - ext, u + ext] */
                double xlo = sp.u - ext - 0.5 - ox, xhi = sp.u + ext - 0.5 - ox;
                double ylo = sp.v - ext - 0.5 - oy, yhi = sp.v + ext - 0.5 - oy;
                int i0 = (int)ceil(xlo / sx), i1 = (int)floor(xhi / sx);
                int j0 = (int)ceil(ylo / sy), j1 = (int)floor(yhi / sy);
                if (i0 < 0) i0 = 0;
                if (j0 < 0) j0 = 0;
                if (i1 > nx - 1) i1 = nx - 1;
                if (j1 > ny - 1) j1 = ny - 1;
                for (int j = j0; j <= j1; ++j)
                    for (int i = i0; i <= i1; ++i) {
                        orc_entry e;
                        e.pix = j * nx + i;
                        e.inst = inst;
                        e.g = g;
                        e.gt = g_off[t] + gl;
                        e.r = sp.r;
                        e.near_ev = near_ev;
                        e.rad_ev = rad_ev;
                        e.valid = sp.valid;
                        e.depth = sp.depth;
                        e.u = sp.u;
                        e.v = sp.v;
                        e.A = sp.conic[0];
                        e.B = sp.conic[1];
                        e.C = sp.conic[2];
                        e.o = sp.opacity;
                        e.rgb[0] = sp.rgb[0];
                        e.rgb[1] = sp.rgb[1];
                        e.rgb[2] = sp.rgb[2];
                        vec_push(vec, &e);
                    }
            }
        }
    }
    /* group entries by pixel (counting sort) */
    size_t npix = (size_t)nx * ny;
    size_t *start = (size_t *)calloc(npix + 1, sizeof(size_t));
    if (!start) return -1;
    size_t total = 0;
    for (int t = 0; t < nthreads; ++t)
        for (size_t k = 0; k < vecs[t].n; ++k) start[vecs[t].e[k].pix + 1]++;
    for (size_t p = 0; p < npix; ++p) start[p + 1] += start[p];
    total = start[npix];
    orc_entry *all = (orc_entry *)malloc((total ? total : 1) * sizeof(orc_entry));
    size_t *cur = (size_t *)malloc((npix + 1) * sizeof(size_t));
    if (!all || !cur) return -1;
    memcpy(cur, start, (npix + 1) * sizeof(size_t));
    for (int t = 0; t < nthreads; ++t) {
        for (size_t k = 0; k < vecs[t].n; ++k) all[cur[vecs[t].e[k].pix]++] = vecs[t].e[k];
        free(vecs[t].e);
    }
    free(vecs);
    free(cur);

    #pragma omp parallel for schedule(dynamic, 64)
    for (long p = 0; p < (long)npix; ++p) {
        orc_entry *L = all + start[p];
        size_t n = start[p + 1] - start[p];
        qsort(L, n, sizeof(orc_entry), cmp_entry);
        int i = (int)(p % nx), j = (int)(p / nx);
        double px = ox + i * sx + 0.5, py = oy + j * sy + 0.5;
        double T = 1.0, C[3] = {0, 0, 0}, ws = 0.0, imp = 0.0;
        uint32_t fl = 0;
        int nc = 0;
        int have_prev = 0;
        double prev_depth = 0, prev_alpha = 0, prev_T = 0, prev_cmax = 0;
        for (size_t k = 0; k < n; ++k) {
            const orc_entry *e = &L[k];
            double dx = px - e->u, dy = py - e->v;
            double q = -0.5 * (e->A * dx * dx + e->C * dy * dy) - e->B * dx * dy;
            double a_raw = e->o * exp(q);
            double alpha = a_raw < 0.99 ? a_raw : 0.99;
            double cmax = dmax(1.0, dmax(e->rgb[0], dmax(e->rgb[1], e->rgb[2])));
            double jump = 2.0 * alpha * T * cmax;
            int live = alpha >= (1.0 / 255.0) * (1.0 - eps->q) && q <= 1e-6;
            int inside = fabs(dx) <= e->r && fabs(dy) <= e->r;
            /* support-box edge close to the centre, or a radius close to an
             * integer with the pixel in the outer ring */
            int near_edge = (fabs(fabs(dx) - e->r) < eps->px && fabs(dy) <= e->r + eps->px) ||
                            (fabs(fabs(dy) - e->r) < eps->px && fabs(dx) <= e->r + eps->px);
            int ring = e->rad_ev && dmax(fabs(dx), fabs(dy)) > e->r - 1.0 - eps->px;
            if ((near_edge || ring) && live) {
                if (jump > eps->impact) fl |= near_edge ? ORC_EV_EDGE : ORC_EV_RADIUS;
                if (jump > imp) imp = jump;
            }
            if ((e->near_ev || lod_ev[e->inst]) && inside && live) {
                if (jump > eps->impact) fl |= e->near_ev ? ORC_EV_NEAR : ORC_EV_LOD;
                if (jump > imp) imp = jump;
            }
            if (!inside || !e->valid) continue;
            if (fabs(q) < 1e-6) {
                double jq = 2.0 * e->o * T * cmax;
                if (jq > eps->impact) fl |= ORC_EV_QZERO;
                if (jq > imp) imp = jq;
            }
            if (q > 0.0) continue;
            /* alpha close to the 1/255 threshold (in the exponent) */
            if (fabs(log(e->o) + q + log(255.0)) < eps->q) {
                double ja = 2.0 * (1.0 / 255.0) * T * cmax;
                if (ja > eps->impact) fl |= ORC_EV_ALPHA;
                if (ja > imp) imp = ja;
            }
            if (alpha < 1.0 / 255.0) continue;
            /* depth near-tie with the previous contributor */
            if (have_prev && fabs(e->depth - prev_depth) < eps->depth_rel * dmax(1.0, fabs(e->depth))) {
                double jt = 2.0 * alpha * prev_alpha * prev_T * dmax(cmax, prev_cmax);
                if (jt > eps->impact) fl |= ORC_EV_TIE;
                if (jt > imp) imp = jt;
            }
            double Tn = T * (1.0 - alpha);
            if (Tn < 1e-4) break;
            for (int ch = 0; ch < 3; ++ch) C[ch] += e->rgb[ch] * alpha * T;
            ws += alpha * T;
            if (contrib) {
                #pragma omp atomic
                contrib[e->gt] += alpha * T;
            }
            have_prev = 1;
            prev_depth = e->depth;
            prev_alpha = alpha;
            prev_T = T;
            prev_cmax = cmax;
            T = Tn;
            ++nc;
        }
        rgba[p * 4 + 0] = C[0];
        rgba[p * 4 + 1] = C[1];
        rgba[p * 4 + 2] = C[2];
        rgba[p * 4 + 3] = 1.0 - T;
        if (wsum) wsum[p] = ws;
        if (flags) flags[p] = fl;
        if (impact) impact[p] = imp;
        if (ncontrib) ncontrib[p] = nc;
    }
    free(all);
    free(start);
    free(lod_ev);
    free(g_off);
    return 0;
}

/* Thread count the oracle runs with (OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
