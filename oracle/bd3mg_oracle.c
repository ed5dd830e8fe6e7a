/*
 * bd3mg_oracle.c -- plain, slow FP64 CPU oracle for the block 3MG (BD3MG)
 * iteration applied to 3D deblurring under depth-variant blur.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  It shares no
 * code, header, table or helper with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Every quantity is computed from its plain definition, in double precision,
 * with no blocking, fusion or algebraic shortcut:
 *   - objective f = f1 + f2 + f3 (Section 3.1, Eq. "crit"):
 *       f1(x) = 1/2 ||Hx - y||^2
 *       f2(x) = eta * sum_n dist(x_n, [xmin, xmax])^2
 *       f3 per penalty mode:
 *         0 (per axis):  lambda * sum_n sum_{a in X,Y,Z} sqrt(delta^2 + ([V^a x]_n)^2)
 *         1 (as printed in Section 3.1): lambda * sum_n sqrt(delta^2 + ([V^X x]_n)^2
 *           + ([V^Y x]_n)^2) + kappa * ||V^Z x||^2;
 *         2 (isotropic over the three axes): lambda * sum_n sqrt(delta^2
 *           + ([V^X x]_n)^2 + ([V^Y x]_n)^2 + ([V^Z x]_n)^2);
 *   - H: depth-variant blur, PSF of the OUTPUT depth, convolution orientation,
 *     zero outside the volume (Eq. "model");
 *   - H^T from the transpose definition (H^T r)_m = sum_n H_{n,m} r_n;
 *   - V^a: forward differences with a zero last row, V^aT from the transpose
 *     definition;
 *   - majorant matrix A(x~) = H^T H + 2 eta I + lambda sum_a V^aT Diag(w_a) V^a,
 *     w_a = 1/sqrt(delta^2 + (V^a x~)^2) (half-quadratic construction the
 *     paper defers to its reference for 3MG, Section 3.1), used in the block
 *     quadratic majorant Q (Section 2.2, Eq. "maj"); in mode 1 the X and Y
 *     differences share the weight w = 1/sqrt(delta^2 + (V^X x~)^2 + (V^Y x~)^2)
 *     and the quadratic Z term contributes its exact Hessian 2 kappa V^ZT V^Z;
 *     in mode 2 all three differences share w = 1/sqrt(delta^2 + sum_a (V^a x~)^2);
 *   - memory-gradient subspace D = [-grad f | d] (Section 2.3), subspace
 *     matrix B = D^T A D by explicit products A*D, u = -B^+ D^T grad f via the
 *     symmetric 2x2 eigendecomposition (Eq. "minimizer", Moore-Penrose
 *     pseudo-inverse), increment D u (Worker box, steps (2)-(6));
 *   - block form: a block S is a slab of depth slices; the restricted step
 *     uses the principal sub-matrix A_(S) (directions zero outside S), and
 *     x_(S) += D_(S) u (Master box, step (2)); blocks are visited in a caller
 *     given order, one after the other (delta = 0, synchronous case of
 *     Section 2.4).
 *
 * Array layout: [nz][ny][nx], x fastest; PSF [nz][pz][py][px] with tap offset
 * a in [-r, r] stored at a + r.  OpenMP (if compiled in) only splits loops over
 * independent output voxels; every per-output sum keeps its order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    int px, py, pz;
    const float *psf;     /* [nz][pz][py][px] */
    double lambda, delta, eta, xmin, xmax;
    int penalty;          /* 0: per-axis hyperbolic; 1: joint X-Y hyperbolic + kappa ||V^Z x||^2;
                             2: isotropic hyperbolic over X, Y, Z */
    double kappa;
} orc_problem;

static long long nvox(const orc_problem *p) { return (long long)p->nx * p->ny * p->nz; }

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* h_z(a, b, c): tap (a, b, c) of the PSF attached to output depth z. */
static double tap(const orc_problem *p, int z, int a, int b, int c) {
    int rx = (p->px - 1) / 2, ry = (p->py - 1) / 2, rz = (p->pz - 1) / 2;
    size_t k = (((size_t)z * p->pz + (size_t)(c + rz)) * p->py + (size_t)(b + ry)) * p->px + (size_t)(a + rx);
    return (double)p->psf[k];
}

/* (Hx)(i,j,z) = sum_{a,b,c} h_z(a,b,c) x(i-a, j-b, z-c), zero outside. */
void orc_apply_H(const orc_problem *p, const double *x, double *out) {
    int rx = (p->px - 1) / 2, ry = (p->py - 1) / 2, rz = (p->pz - 1) / 2;
    int z;
#pragma omp parallel for schedule(dynamic)
    for (z = 0; z < p->nz; ++z)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                double s = 0.0;
                for (int c = -rz; c <= rz; ++c) {
                    int zs = z - c;
                    if (zs < 0 || zs >= p->nz) continue;
                    for (int b = -ry; b <= ry; ++b) {
                        int js = j - b;
                        if (js < 0 || js >= p->ny) continue;
                        for (int a = -rx; a <= rx; ++a) {
                            int is = i - a;
                            if (is < 0 || is >= p->nx) continue;
                            s += tap(p, z, a, b, c) * x[((size_t)zs * p->ny + js) * p->nx + is];
                        }
                    }
                }
                out[((size_t)z * p->ny + j) * p->nx + i] = s;
            }
}

/* (H^T r)_m = sum_n H_{n,m} r_n with H_{n,m} = h_{z_n}(i_n-i_m, j_n-j_m, z_n-z_m):
 * every output voxel n that the input voxel m contributes to. */
void orc_apply_HT(const orc_problem *p, const double *r, double *out) {
    int rx = (p->px - 1) / 2, ry = (p->py - 1) / 2, rz = (p->pz - 1) / 2;
    int zm;
#pragma omp parallel for schedule(dynamic)
    for (zm = 0; zm < p->nz; ++zm)
        for (int jm = 0; jm < p->ny; ++jm)
            for (int im = 0; im < p->nx; ++im) {
                double s = 0.0;
                for (int c = -rz; c <= rz; ++c) {
                    int zn = zm + c;
                    if (zn < 0 || zn >= p->nz) continue;
                    for (int b = -ry; b <= ry; ++b) {
                        int jn = jm + b;
                        if (jn < 0 || jn >= p->ny) continue;
                        for (int a = -rx; a <= rx; ++a) {
                            int in = im + a;
                            if (in < 0 || in >= p->nx) continue;
                            s += tap(p, zn, a, b, c) * r[((size_t)zn * p->ny + jn) * p->nx + in];
                        }
                    }
                }
                out[((size_t)zm * p->ny + jm) * p->nx + im] = s;
            }
}

/* Forward difference along axis (0 = X, 1 = Y, 2 = Z), zero on the last plane. */
void orc_apply_V(const orc_problem *p, int axis, const double *x, double *out) {
    long long n = nvox(p);
    long long stride = axis == 0 ? 1 : axis == 1 ? p->nx : (long long)p->nx * p->ny;
    for (long long k = 0; k < n; ++k) {
        int i = (int)(k % p->nx), j = (int)((k / p->nx) % p->ny), z = (int)(k / ((long long)p->nx * p->ny));
        int pos = axis == 0 ? i : axis == 1 ? j : z;
        int len = axis == 0 ? p->nx : axis == 1 ? p->ny : p->nz;
        out[k] = (pos < len - 1) ? x[k + stride] - x[k] : 0.0;
    }
}

/* (V^T q)_m = sum_n V_{n,m} q_n: +q_{m-e} from row m-e (if m-e exists and is
 * not on the last plane, which holds whenever it exists), -q_m from row m (if m
 * is not on the last plane). */
void orc_apply_VT(const orc_problem *p, int axis, const double *q, double *out) {
    long long n = nvox(p);
    long long stride = axis == 0 ? 1 : axis == 1 ? p->nx : (long long)p->nx * p->ny;
    for (long long k = 0; k < n; ++k) {
        int i = (int)(k % p->nx), j = (int)((k / p->nx) % p->ny), z = (int)(k / ((long long)p->nx * p->ny));
        int pos = axis == 0 ? i : axis == 1 ? j : z;
        int len = axis == 0 ? p->nx : axis == 1 ? p->ny : p->nz;
        double s = 0.0;
        if (pos >= 1) s += q[k - stride];
        if (pos < len - 1) s -= q[k];
        out[k] = s;
    }
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* f(x) with its three parts: parts[0] = f1, parts[1] = f2 (box), parts[2] = f3. */
double orc_objective(const orc_problem *p, const float *y, const double *x, double *parts) {
    long long n = nvox(p);
    double *hx = (double *)malloc(sizeof(double) * n);
    double *t = (double *)malloc(sizeof(double) * n);
    orc_apply_H(p, x, hx);
    double f1 = 0.0, f2 = 0.0, f3 = 0.0;
    for (long long k = 0; k < n; ++k) {
        double r = hx[k] - (double)y[k];
        f1 += 0.5 * r * r;
    }
    for (long long k = 0; k < n; ++k) {
        double dist = x[k] - clampd(x[k], p->xmin, p->xmax);
        f2 += p->eta * dist * dist;
    }
    if (p->penalty == 0) {
        for (int axis = 0; axis < 3; ++axis) {
            orc_apply_V(p, axis, x, t);
            for (long long k = 0; k < n; ++k) f3 += p->lambda * sqrt(p->delta * p->delta + t[k] * t[k]);
        }
    } else if (p->penalty == 1) {
        double *ty = (double *)malloc(sizeof(double) * n);
        orc_apply_V(p, 0, x, t);
        orc_apply_V(p, 1, x, ty);
        for (long long k = 0; k < n; ++k) f3 += p->lambda * sqrt(p->delta * p->delta + t[k] * t[k] + ty[k] * ty[k]);
        orc_apply_V(p, 2, x, t);
        for (long long k = 0; k < n; ++k) f3 += p->kappa * t[k] * t[k];
        free(ty);
    } else {
        double *ty = (double *)malloc(sizeof(double) * n);
        double *tz = (double *)malloc(sizeof(double) * n);
        orc_apply_V(p, 0, x, t);
        orc_apply_V(p, 1, x, ty);
        orc_apply_V(p, 2, x, tz);
        for (long long k = 0; k < n; ++k)
            f3 += p->lambda * sqrt(p->delta * p->delta + t[k] * t[k] + ty[k] * ty[k] + tz[k] * tz[k]);
        free(ty);
        free(tz);
    }
    free(hx);
    free(t);
    if (parts) { parts[0] = f1; parts[1] = f2; parts[2] = f3; }
    return f1 + f2 + f3;
}

/* grad f(x) = H^T(Hx - y) + 2 eta (x - P(x)) + the penalty's gradient:
 *   mode 0: lambda sum_a V^aT psi'(V^a x), psi'(t) = t / sqrt(delta^2 + t^2);
 *   mode 1: lambda (V^XT (w t_X) + V^YT (w t_Y)) + 2 kappa V^ZT V^Z x,
 *           t_a = V^a x, w = 1/sqrt(delta^2 + t_X^2 + t_Y^2);
 *   mode 2: lambda sum_a V^aT (w t_a), w = 1/sqrt(delta^2 + t_X^2 + t_Y^2 + t_Z^2). */
void orc_gradient(const orc_problem *p, const float *y, const double *x, double *g) {
    long long n = nvox(p);
    double *r = (double *)malloc(sizeof(double) * n);
    double *t = (double *)malloc(sizeof(double) * n);
    double *vt = (double *)malloc(sizeof(double) * n);
    orc_apply_H(p, x, r);
    for (long long k = 0; k < n; ++k) r[k] -= (double)y[k];
    orc_apply_HT(p, r, g);
    for (long long k = 0; k < n; ++k) g[k] += 2.0 * p->eta * (x[k] - clampd(x[k], p->xmin, p->xmax));
    if (p->penalty == 0) {
        for (int axis = 0; axis < 3; ++axis) {
            orc_apply_V(p, axis, x, t);
            for (long long k = 0; k < n; ++k) t[k] = t[k] / sqrt(p->delta * p->delta + t[k] * t[k]);
            orc_apply_VT(p, axis, t, vt);
            for (long long k = 0; k < n; ++k) g[k] += p->lambda * vt[k];
        }
    } else if (p->penalty == 2) {
        double *ta[3], *w = (double *)malloc(sizeof(double) * n);
        for (int axis = 0; axis < 3; ++axis) {
            ta[axis] = (double *)malloc(sizeof(double) * n);
            orc_apply_V(p, axis, x, ta[axis]);
        }
        for (long long k = 0; k < n; ++k)
            w[k] = 1.0 / sqrt(p->delta * p->delta + ta[0][k] * ta[0][k] + ta[1][k] * ta[1][k] + ta[2][k] * ta[2][k]);
        for (int axis = 0; axis < 3; ++axis) {
            for (long long k = 0; k < n; ++k) ta[axis][k] *= w[k];
            orc_apply_VT(p, axis, ta[axis], vt);
            for (long long k = 0; k < n; ++k) g[k] += p->lambda * vt[k];
            free(ta[axis]);
        }
        free(w);
    } else {
        double *ty = (double *)malloc(sizeof(double) * n);
        orc_apply_V(p, 0, x, t);
        orc_apply_V(p, 1, x, ty);
        for (long long k = 0; k < n; ++k) {
            double w = 1.0 / sqrt(p->delta * p->delta + t[k] * t[k] + ty[k] * ty[k]);
            t[k] *= w;
            ty[k] *= w;
        }
        orc_apply_VT(p, 0, t, vt);
        for (long long k = 0; k < n; ++k) g[k] += p->lambda * vt[k];
        orc_apply_VT(p, 1, ty, vt);
        for (long long k = 0; k < n; ++k) g[k] += p->lambda * vt[k];
        orc_apply_V(p, 2, x, t);
        orc_apply_VT(p, 2, t, vt);
        for (long long k = 0; k < n; ++k) g[k] += 2.0 * p->kappa * vt[k];
        free(ty);
    }
    free(r);
    free(t);
    free(vt);
}

/* A(xt) v = H^T H v + 2 eta v + the penalty's majorant curvature:
 *   mode 0: lambda sum_a V^aT (w_a * V^a v), w_a = 1/sqrt(delta^2 + (V^a xt)^2);
 *   mode 1: lambda (V^XT (w V^X v) + V^YT (w V^Y v)) + 2 kappa V^ZT V^Z v,
 *           w = 1/sqrt(delta^2 + (V^X xt)^2 + (V^Y xt)^2);
 *   mode 2: lambda sum_a V^aT (w V^a v), w = 1/sqrt(delta^2 + sum_a (V^a xt)^2). */
void orc_apply_A(const orc_problem *p, const double *xt, const double *v, double *out) {
    long long n = nvox(p);
    double *hv = (double *)malloc(sizeof(double) * n);
    double *tx = (double *)malloc(sizeof(double) * n);
    double *tv = (double *)malloc(sizeof(double) * n);
    double *vt = (double *)malloc(sizeof(double) * n);
    orc_apply_H(p, v, hv);
    orc_apply_HT(p, hv, out);
    for (long long k = 0; k < n; ++k) out[k] += 2.0 * p->eta * v[k];
    if (p->penalty == 0) {
        for (int axis = 0; axis < 3; ++axis) {
            orc_apply_V(p, axis, xt, tx);
            orc_apply_V(p, axis, v, tv);
            for (long long k = 0; k < n; ++k) tv[k] *= 1.0 / sqrt(p->delta * p->delta + tx[k] * tx[k]);
            orc_apply_VT(p, axis, tv, vt);
            for (long long k = 0; k < n; ++k) out[k] += p->lambda * vt[k];
        }
    } else if (p->penalty == 2) {
        double *w = (double *)malloc(sizeof(double) * n);
        for (long long k = 0; k < n; ++k) w[k] = p->delta * p->delta;
        for (int axis = 0; axis < 3; ++axis) {
            orc_apply_V(p, axis, xt, tx);
            for (long long k = 0; k < n; ++k) w[k] += tx[k] * tx[k];
        }
        for (long long k = 0; k < n; ++k) w[k] = 1.0 / sqrt(w[k]);
        for (int axis = 0; axis < 3; ++axis) {
            orc_apply_V(p, axis, v, tv);
            for (long long k = 0; k < n; ++k) tv[k] *= w[k];
            orc_apply_VT(p, axis, tv, vt);
            for (long long k = 0; k < n; ++k) out[k] += p->lambda * vt[k];
        }
        free(w);
    } else {
        double *ty = (double *)malloc(sizeof(double) * n);
        double *w = (double *)malloc(sizeof(double) * n);
        orc_apply_V(p, 0, xt, tx);
        orc_apply_V(p, 1, xt, ty);
        for (long long k = 0; k < n; ++k) w[k] = 1.0 / sqrt(p->delta * p->delta + tx[k] * tx[k] + ty[k] * ty[k]);
        for (int axis = 0; axis < 2; ++axis) {
            orc_apply_V(p, axis, v, tv);
            for (long long k = 0; k < n; ++k) tv[k] *= w[k];
            orc_apply_VT(p, axis, tv, vt);
            for (long long k = 0; k < n; ++k) out[k] += p->lambda * vt[k];
        }
        orc_apply_V(p, 2, v, tv);
        orc_apply_VT(p, 2, tv, vt);
        for (long long k = 0; k < n; ++k) out[k] += 2.0 * p->kappa * vt[k];
        free(ty);
        free(w);
    }
    free(hv);
    free(tx);
    free(tv);
    free(vt);
}

/* u = -B^+ c for a symmetric 2x2 B = [[b00, b01], [b01, b11]] (row-major B[4]),
 * via its eigendecomposition; eigenvalues <= rtol * (largest |eigenvalue|)
 * are treated as zero (Moore-Penrose pseudo-inverse).  Returns the rank used. */
int orc_pinv2_solve(const double *B, const double *c, double *u, double rtol) {
    double a = B[0], b = 0.5 * (B[1] + B[2]), d = B[3];
    double tr = a + d, diff = a - d;
    double disc = sqrt(diff * diff + 4.0 * b * b);
    double l[2] = {0.5 * (tr + disc), 0.5 * (tr - disc)};
    double vec[2][2];
    /* eigenvector for l[0]: (b, l0 - a) or (l0 - d, b); pick the better conditioned. */
    for (int e = 0; e < 2; ++e) {
        double v0 = b, v1 = l[e] - a;
        double w0 = l[e] - d, w1 = b;
        double nv = hypot(v0, v1), nw = hypot(w0, w1);
        if (nv >= nw && nv > 0) { vec[e][0] = v0 / nv; vec[e][1] = v1 / nv; }
        else if (nw > 0) { vec[e][0] = w0 / nw; vec[e][1] = w1 / nw; }
        else { vec[e][0] = e == 0 ? 1.0 : 0.0; vec[e][1] = e == 0 ? 0.0 : 1.0; }
    }
    if (disc == 0.0) { vec[0][0] = 1; vec[0][1] = 0; vec[1][0] = 0; vec[1][1] = 1; }
    double lmax = fmax(fabs(l[0]), fabs(l[1]));
    u[0] = 0.0; u[1] = 0.0;
    int rank = 0;
    for (int e = 0; e < 2; ++e) {
        if (lmax <= 0.0 || fabs(l[e]) <= rtol * lmax) continue;
        double proj = vec[e][0] * c[0] + vec[e][1] * c[1];
        u[0] -= proj / l[e] * vec[e][0];
        u[1] -= proj / l[e] * vec[e][1];
        ++rank;
    }
    return rank;
}

static double dot(const double *a, const double *b, long long n) {
    double s = 0.0;
    for (long long k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* One restricted 3MG step on the slab of depth slices [z0, z1) (whole volume if
 * z0 = 0, z1 = nz): D = [-g_S | d_S], B = D^T A(x) D, c = D^T g, u = -B^+ c,
 * x_S += D u, d_S = D u.  info (optional, 8 doubles): B[4], c[2], u[2]. */
void orc_3mg_step(const orc_problem *p, const float *y, double *x, double *d, int z0, int z1,
                  double pinv_rtol, double *info) {
    long long n = nvox(p);
    long long plane = (long long)p->nx * p->ny;
    long long k0 = (long long)z0 * plane, k1 = (long long)z1 * plane;
    double *g = (double *)calloc(n, sizeof(double));
    double *D0 = (double *)calloc(n, sizeof(double));
    double *D1 = (double *)calloc(n, sizeof(double));
    double *A0 = (double *)malloc(sizeof(double) * n);
    double *A1 = (double *)malloc(sizeof(double) * n);
    orc_gradient(p, y, x, g);
    for (long long k = k0; k < k1; ++k) { D0[k] = -g[k]; D1[k] = d[k]; }
    orc_apply_A(p, x, D0, A0);
    orc_apply_A(p, x, D1, A1);
    double B[4] = {dot(D0, A0, n), dot(D0, A1, n), dot(D1, A0, n), dot(D1, A1, n)};
    double gS[2] = {0, 0};
    for (long long k = k0; k < k1; ++k) { gS[0] += D0[k] * g[k]; gS[1] += D1[k] * g[k]; }
    double u[2];
    orc_pinv2_solve(B, gS, u, pinv_rtol);
    for (long long k = k0; k < k1; ++k) {
        double inc = u[0] * D0[k] + u[1] * D1[k];
        x[k] += inc;
        d[k] = inc;
    }
    if (info) {
        info[0] = B[0]; info[1] = B[1]; info[2] = B[2]; info[3] = B[3];
        info[4] = gS[0]; info[5] = gS[1]; info[6] = u[0]; info[7] = u[1];
    }
    free(g); free(D0); free(D1); free(A0); free(A1);
}

/* n_sweeps sweeps; each sweep visits the slabs order[0..nslabs-1] one after the
 * other (bounds: nslabs+1 slice indices).  f_trace (n_sweeps + 1 entries,
 * optional) receives f(x^k) before sweep k and after the last one. */
void orc_3mg(const orc_problem *p, const float *y, double *x, double *d, int n_sweeps, int nslabs,
             const int *bounds, const int *order, double pinv_rtol, double *f_trace) {
    for (int k = 0; k < n_sweeps; ++k) {
        if (f_trace) f_trace[k] = orc_objective(p, y, x, NULL);
        for (int s = 0; s < nslabs; ++s) {
            int b = order ? order[s] : s;
            orc_3mg_step(p, y, x, d, bounds[b], bounds[b + 1], pinv_rtol, NULL);
        }
    }
    if (f_trace) f_trace[n_sweeps] = orc_objective(p, y, x, NULL);
}

/* Gradient at selected voxels only, each from its plain local definition:
 * [H^T r]_m needs r_n = (Hx)_n - y_n at the voxels n that m feeds. */
void orc_gradient_at(const orc_problem *p, const float *y, const double *x, int count,
                     const long long *idx, double *out) {
    int rx = (p->px - 1) / 2, ry = (p->py - 1) / 2, rz = (p->pz - 1) / 2;
    int q;
#pragma omp parallel for schedule(dynamic)
    for (q = 0; q < count; ++q) {
        long long m = idx[q];
        int im = (int)(m % p->nx), jm = (int)((m / p->nx) % p->ny), zm = (int)(m / ((long long)p->nx * p->ny));
        double s = 0.0;
        for (int c = -rz; c <= rz; ++c) {
            int zn = zm + c;
            if (zn < 0 || zn >= p->nz) continue;
            for (int b = -ry; b <= ry; ++b) {
                int jn = jm + b;
                if (jn < 0 || jn >= p->ny) continue;
                for (int a = -rx; a <= rx; ++a) {
                    int in = im + a;
                    if (in < 0 || in >= p->nx) continue;
                    /* r_n = (Hx)_n - y_n */
                    double hx = 0.0;
                    for (int c2 = -rz; c2 <= rz; ++c2) {
                        int zs = zn - c2;
                        if (zs < 0 || zs >= p->nz) continue;
                        for (int b2 = -ry; b2 <= ry; ++b2) {
                            int js = jn - b2;
                            if (js < 0 || js >= p->ny) continue;
                            for (int a2 = -rx; a2 <= rx; ++a2) {
                                int is = in - a2;
                                if (is < 0 || is >= p->nx) continue;
                                hx += tap(p, zn, a2, b2, c2) * x[((size_t)zs * p->ny + js) * p->nx + is];
                            }
                        }
                    }
                    double r = hx - (double)y[((size_t)zn * p->ny + jn) * p->nx + in];
                    s += tap(p, zn, a, b, c) * r;
                }
            }
        }
        double xm = x[m];
        s += 2.0 * p->eta * (xm - clampd(xm, p->xmin, p->xmax));
        int pos[3] = {im, jm, zm};
        int len[3] = {p->nx, p->ny, p->nz};
        long long stride[3] = {1, p->nx, (long long)p->nx * p->ny};
        if (p->penalty == 0) {
            /* penalty: lambda * sum_a [psi'(t_a at m - e_a) - psi'(t_a at m)] */
            for (int axis = 0; axis < 3; ++axis) {
                if (pos[axis] >= 1) {
                    double t = xm - x[m - stride[axis]];
                    s += p->lambda * t / sqrt(p->delta * p->delta + t * t);
                }
                if (pos[axis] < len[axis] - 1) {
                    double t = x[m + stride[axis]] - xm;
                    s -= p->lambda * t / sqrt(p->delta * p->delta + t * t);
                }
            }
        } else if (p->penalty == 2) {
            /* isotropic term: lambda * [sum_a w t_a at m - e_a - w (t_X + t_Y + t_Z) at m], with
             * t_a, w of a voxel from its own forward differences */
            for (int e = 0; e < 4; ++e) {
                if (e > 0 && pos[e - 1] < 1) continue;
                long long v = e == 0 ? m : m - stride[e - 1];
                int pv[3] = {(int)(v % p->nx), (int)((v / p->nx) % p->ny), (int)(v / stride[2])};
                double ta[3], ss = p->delta * p->delta;
                for (int axis = 0; axis < 3; ++axis) {
                    ta[axis] = pv[axis] < len[axis] - 1 ? x[v + stride[axis]] - x[v] : 0.0;
                    ss += ta[axis] * ta[axis];
                }
                double w = 1.0 / sqrt(ss);
                if (e == 0) s -= p->lambda * w * (ta[0] + ta[1] + ta[2]);
                else s += p->lambda * w * ta[e - 1];
            }
        } else {
            /* joint X-Y term: lambda * [w t_X at m - e_X + w t_Y at m - e_Y - w (t_X + t_Y) at m],
             * with t_a, w of a voxel from its own forward differences; Z term: 2 kappa V^ZT V^Z x */
            long long at[3] = {m, im >= 1 ? m - 1 : -1, jm >= 1 ? m - p->nx : -1};
            for (int e = 0; e < 3; ++e) {
                long long v = at[e];
                if (v < 0) continue;
                int iv = (int)(v % p->nx), jv = (int)((v / p->nx) % p->ny);
                double tx = iv < p->nx - 1 ? x[v + 1] - x[v] : 0.0;
                double ty = jv < p->ny - 1 ? x[v + p->nx] - x[v] : 0.0;
                double w = 1.0 / sqrt(p->delta * p->delta + tx * tx + ty * ty);
                if (e == 0) s -= p->lambda * w * (tx + ty);
                else if (e == 1) s += p->lambda * w * tx;
                else s += p->lambda * w * ty;
            }
            if (pos[2] >= 1) s += 2.0 * p->kappa * (xm - x[m - stride[2]]);
            if (pos[2] < len[2] - 1) s -= 2.0 * p->kappa * (x[m + stride[2]] - xm);
        }
        out[q] = s;
    }
}

/* ------------------------------------------------------------------------
 * Ablation variants of Section 3.2 (Table 1) and the block schedules.
 *
 *   metric 0: the half-quadratic majorant A(x) above (3MG, BD3MG, BP3MG);
 *   metric 1: A = L I, L a bound on the Lipschitz constant of grad f
 *             (Async-GD, Async-CG);
 *   direction 0: D = [-g | d] (memory gradient, 2x2 solve);
 *   direction 1: D = -g (gradient only, 1x1 solve; Async-GD);
 *   direction 2: conjugate direction p = -g + beta p_prev with the
 *             Fletcher-Reeves beta = ||g||^2 / ||g_prev||^2 of the block, and
 *             the step minimising the block majorant along p (the closed-form
 *             stepsize of memory-gradient / CG methods), restarted with
 *             p = -g when p is not a descent direction (Async-CG);
 *   schedule 0: blocks one after the other in the given order (delta = 0);
 *   schedule 1: Jacobi -- every block's step computed from the same iterate
 *             x^k and all of them added (the parallel block update of BP3MG);
 *   inflation: the block majorant's curvature scaled by this factor >= 1
 *             (Assumption C asks the block curvature to exceed the delayed
 *             one; m blocks updated at once from the same iterate majorise f
 *             when it is at least m, by (sum_S v_S)^T A (sum_S v_S) <=
 *             m sum_S v_S^T A v_S for positive semidefinite A).
 * ------------------------------------------------------------------------ */
typedef struct {
    int metric;
    double lipschitz;
    int direction;
    int schedule;
    double inflation;
} orc_variant;

/* Upper bound on the Lipschitz constant of grad f: ||H||_2^2 <= ||H||_1 ||H||_inf
 * (largest absolute column sum times largest absolute row sum of H), the box
 * term's 2 eta, and the penalty's Hessian bound (its curvature in t is at most
 * lambda / delta, ||V^a||_2 <= 2): mode 0 and mode 2, 12 lambda / delta;
 * mode 1, 8 lambda / delta + 8 kappa. */
double orc_lipschitz_bound(const orc_problem *p) {
    int rx = (p->px - 1) / 2, ry = (p->py - 1) / 2, rz = (p->pz - 1) / 2;
    double rowmax = 0.0, colmax = 0.0;
    for (int z = 0; z < p->nz; ++z) {
        double s = 0.0;
        for (int c = -rz; c <= rz; ++c)
            for (int b = -ry; b <= ry; ++b)
                for (int a = -rx; a <= rx; ++a) s += fabs(tap(p, z, a, b, c));
        if (s > rowmax) rowmax = s;
    }
    /* column of input depth zi: every output depth z = zi + c that reads it */
    for (int zi = 0; zi < p->nz; ++zi) {
        double s = 0.0;
        for (int c = -rz; c <= rz; ++c) {
            int z = zi + c;
            if (z < 0 || z >= p->nz) continue;
            for (int b = -ry; b <= ry; ++b)
                for (int a = -rx; a <= rx; ++a) s += fabs(tap(p, z, a, b, c));
        }
        if (s > colmax) colmax = s;
    }
    double pen = p->penalty == 1 ? 8.0 * p->lambda / p->delta + 8.0 * p->kappa : 12.0 * p->lambda / p->delta;
    return rowmax * colmax + 2.0 * p->eta + pen;
}

/* One block step of a variant on the slab [z0, z1): g and the metric are taken
 * at xe (the sweep's iterate for the Jacobi schedule, x itself otherwise); the
 * increment D u is added to x and stored in d.  state[2] carries the block's
 * previous ||g_S||^2 and step length for direction 2 (zero at the start).
 * info (optional, 8): B[4], c[2], u[2]. */
void orc_3mg_step_v(const orc_problem *p, const orc_variant *v, const float *y, const double *xe, double *x,
                    double *d, int z0, int z1, double pinv_rtol, double *state, double *info) {
    long long n = nvox(p);
    long long plane = (long long)p->nx * p->ny;
    long long k0 = (long long)z0 * plane, k1 = (long long)z1 * plane;
    double *g = (double *)calloc(n, sizeof(double));
    double *D0 = (double *)calloc(n, sizeof(double));
    double *D1 = (double *)calloc(n, sizeof(double));
    double *A0 = (double *)malloc(sizeof(double) * n);
    double *A1 = (double *)malloc(sizeof(double) * n);
    orc_gradient(p, y, xe, g);
    for (long long k = k0; k < k1; ++k) { D0[k] = -g[k]; D1[k] = v->direction == 1 ? 0.0 : d[k]; }
    if (v->metric == 1) {
        for (long long k = 0; k < n; ++k) { A0[k] = v->lipschitz * D0[k]; A1[k] = v->lipschitz * D1[k]; }
    } else {
        orc_apply_A(p, xe, D0, A0);
        orc_apply_A(p, xe, D1, A1);
    }
    double B[4] = {dot(D0, A0, n), dot(D0, A1, n), dot(D1, A0, n), dot(D1, A1, n)};
    for (int i = 0; i < 4; ++i) B[i] *= v->inflation;
    double gS[2] = {0, 0};
    for (long long k = k0; k < k1; ++k) { gS[0] += D0[k] * g[k]; gS[1] += D1[k] * g[k]; }
    double u[2] = {0.0, 0.0};
    if (v->direction == 0) {
        orc_pinv2_solve(B, gS, u, pinv_rtol);
    } else if (v->direction == 1) {
        if (B[0] > 0.0) u[0] = -gS[0] / B[0];
    } else {
        /* p = -g + beta p_prev, p_prev = d / (previous step): p = D [1, beta'] */
        double gg = -gS[0], bp = 0.0;
        if (state[0] > 0.0 && state[1] > 0.0) bp = (gg / state[0]) / state[1];
        double slope = gS[0] + bp * gS[1];
        double curv = B[0] + bp * (B[1] + B[2]) + bp * bp * B[3];
        if (!(slope < 0.0) || !(curv > 0.0)) {             /* restart along -g */
            bp = 0.0;
            slope = gS[0];
            curv = B[0];
        }
        if (curv > 0.0) {
            double a = -slope / curv;
            u[0] = a;
            u[1] = a * bp;
        }
        state[0] = gg;
        state[1] = u[0];
    }
    for (long long k = k0; k < k1; ++k) {
        double inc = u[0] * D0[k] + u[1] * D1[k];
        x[k] += inc;
        d[k] = inc;
    }
    if (info) {
        info[0] = B[0]; info[1] = B[1]; info[2] = B[2]; info[3] = B[3];
        info[4] = gS[0]; info[5] = gS[1]; info[6] = u[0]; info[7] = u[1];
    }
    free(g); free(D0); free(D1); free(A0); free(A1);
}

/* n_sweeps sweeps of a variant: schedule 0 visits the slabs order[0..nslabs-1]
 * one after the other; schedule 1 computes every slab's step from the sweep's
 * iterate and adds them all.  state: 2 * nslabs doubles (direction 2), zero at
 * the start.  f_trace (optional, n_sweeps + 1) as in orc_3mg. */
void orc_3mg_v(const orc_problem *p, const orc_variant *v, const float *y, double *x, double *d, int n_sweeps,
               int nslabs, const int *bounds, const int *order, double pinv_rtol, double *state, double *f_trace) {
    long long n = nvox(p);
    double *xk = (double *)malloc(sizeof(double) * n);
    for (int k = 0; k < n_sweeps; ++k) {
        if (f_trace) f_trace[k] = orc_objective(p, y, x, NULL);
        if (v->schedule == 1) memcpy(xk, x, sizeof(double) * n);
        for (int s = 0; s < nslabs; ++s) {
            int b = order ? order[s] : s;
            orc_3mg_step_v(p, v, y, v->schedule == 1 ? xk : x, x, d, bounds[b], bounds[b + 1], pinv_rtol,
                           state + 2 * b, NULL);
        }
    }
    if (f_trace) f_trace[n_sweeps] = orc_objective(p, y, x, NULL);
    free(xk);
}
