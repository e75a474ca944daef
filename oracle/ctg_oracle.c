/*
 * FP64 CPU oracle for the two CT projectors of the unmatched pair (A, B).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * library.
 *
 * The paper (Sec. 1, eq. (1.1)-(1.2)) fixes the roles: A in R^{m x n} is the
 * forward projector, B in R^{n x m} an unmatched back projector, m = N_a*N_d,
 * n = N^2.  Sec. 6.1 names the interpolation ("Joseph") model for A but gives
 * no formulas; the discretisation below is this project's reading of it:
 *
 *   grid     pixel (i, j) centre (x_j, y_i) = (j - h, i - h), h = (N-1)/2;
 *            angle theta_a = S + a*R/N_a degrees (integers S, R, endpoint
 *            excluded); detector centre s_d = (d - (N_d-1)/2) * ds;
 *            ray (a, d) = { (x, y) : x cos + y sin = s_d }.
 *   A        Joseph: a ray is "row-driven" iff theta mod 180 lies in
 *            [0, 45] or [135, 180) (decided on integers, so 45 and 135 are
 *            row-driven).  Row-driven: per row i, u = (s_d - y_i sin)/cos + h,
 *            linear interpolation between x[i, floor(u)] and x[i, floor(u)+1]
 *            (out-of-image taps are 0), the sum scaled by 1/|cos|.
 *            Column-driven: per column j, v = (s_d - x_j cos)/sin + h,
 *            interpolation down column j, sum scaled by 1/|sin|.
 *   B        pixel-driven: (B b)[i, j] = sum_a (1-f) b[a, d0] + f b[a, d0+1],
 *            u = (x_j cos + y_i sin)/ds + (N_d-1)/2, d0 = floor(u), f = u - d0,
 *            out-of-range bins contribute 0.
 *
 * cos/sin are evaluated in FP64 and set exactly to 0 or +-1 at multiples of
 * 90 degrees.  Every routine returns 0 on success, -1 on an invalid geometry.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    int N, n_angles, n_det;
    double start_deg, range_deg, ds;
} geom_t;

static int geom_ok(const geom_t *g) {
    if (g->N < 1 || g->n_angles < 1 || g->n_det < 1) return 0;
    if (!(g->ds > 0.0)) return 0;
    if (g->start_deg != floor(g->start_deg)) return 0;
    if (g->range_deg != floor(g->range_deg) || g->range_deg <= 0.0) return 0;
    return 1;
}

/* theta_a in degrees is num/N_a with the integer num = S*N_a + a*R. */
static void angle(const geom_t *g, int a, double *c, double *s, int *row_driven) {
    const int64_t Na = g->n_angles;
    const int64_t num = (int64_t)g->start_deg * Na + (int64_t)a * (int64_t)g->range_deg;
    const int64_t P = 180 * Na;
    int64_t T = num % P;
    if (T < 0) T += P;
    *row_driven = (4 * T <= P) || (4 * T >= 3 * P);
    const int64_t Q = 90 * Na;
    if (num % Q == 0) {
        int64_t k = (num / Q) % 4;
        if (k < 0) k += 4;
        const double cc[4] = {1.0, 0.0, -1.0, 0.0};
        const double ss[4] = {0.0, 1.0, 0.0, -1.0};
        *c = cc[k];
        *s = ss[k];
    } else {
        const double th = (double)num * M_PI / (double)P;
        *c = cos(th);
        *s = sin(th);
    }
}

int orc_angles(int N, int Na, int Nd, double S, double R, double ds,
               double *cos_out, double *sin_out, int32_t *row_driven) {
    geom_t g = {N, Na, Nd, S, R, ds};
    if (!geom_ok(&g)) return -1;
    for (int a = 0; a < Na; ++a) {
        int rd;
        angle(&g, a, &cos_out[a], &sin_out[a], &rd);
        row_driven[a] = rd;
    }
    return 0;
}

/* b = A x.  x: N*N row-major, b: N_a*N_d angle-major. */
int orc_forward(int N, int Na, int Nd, double S, double R, double ds,
                const double *x, double *b) {
    geom_t g = {N, Na, Nd, S, R, ds};
    if (!geom_ok(&g)) return -1;
    const double h = 0.5 * (N - 1), hd = 0.5 * (Nd - 1);
#pragma omp parallel for schedule(static)
    for (long ray = 0; ray < (long)Na * Nd; ++ray) {
        const int a = (int)(ray / Nd), d = (int)(ray % Nd);
        double c, s;
        int rd;
        angle(&g, a, &c, &s, &rd);
        const double sd = (d - hd) * ds;
        double acc = 0.0;
        if (rd) {
            for (int i = 0; i < N; ++i) {
                const double u = (sd - (i - h) * s) / c + h;
                const double fl = floor(u);
                const long j0 = (long)fl;
                const double f = u - fl;
                if (j0 >= 0 && j0 < N) acc += (1.0 - f) * x[(long)i * N + j0];
                if (j0 + 1 >= 0 && j0 + 1 < N) acc += f * x[(long)i * N + j0 + 1];
            }
            acc /= fabs(c);
        } else {
            for (int j = 0; j < N; ++j) {
                const double v = (sd - (j - h) * c) / s + h;
                const double fl = floor(v);
                const long i0 = (long)fl;
                const double f = v - fl;
                if (i0 >= 0 && i0 < N) acc += (1.0 - f) * x[i0 * N + j];
                if (i0 + 1 >= 0 && i0 + 1 < N) acc += f * x[(i0 + 1) * N + j];
            }
            acc /= fabs(s);
        }
        b[ray] = acc;
    }
    return 0;
}

/* x = B b (pixel-driven, gather over angles). */
int orc_backproject(int N, int Na, int Nd, double S, double R, double ds,
                    const double *b, double *x) {
    geom_t g = {N, Na, Nd, S, R, ds};
    if (!geom_ok(&g)) return -1;
    const double h = 0.5 * (N - 1), hd = 0.5 * (Nd - 1);
    double *cs = (double *)malloc(sizeof(double) * 2 * Na);
    if (!cs) return -1;
    for (int a = 0; a < Na; ++a) {
        int rd;
        angle(&g, a, &cs[2 * a], &cs[2 * a + 1], &rd);
    }
#pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)N * N; ++p) {
        const int i = (int)(p / N), j = (int)(p % N);
        const double xj = j - h, yi = i - h;
        double acc = 0.0;
        for (int a = 0; a < Na; ++a) {
            const double u = (xj * cs[2 * a] + yi * cs[2 * a + 1]) / ds + hd;
            const double fl = floor(u);
            const long d0 = (long)fl;
            const double f = u - fl;
            if (d0 >= 0 && d0 < Nd) acc += (1.0 - f) * b[(long)a * Nd + d0];
            if (d0 + 1 >= 0 && d0 + 1 < Nd) acc += f * b[(long)a * Nd + d0 + 1];
        }
        x[p] = acc;
    }
    free(cs);
    return 0;
}

/* Explicit A as (row, col, val) triplets; zero weights are skipped.
 * Capacity needed: 2 * N_a * N_d * N.  Returns the count, or -1. */
long orc_forward_triplets(int N, int Na, int Nd, double S, double R, double ds,
                          int64_t *rows, int64_t *cols, double *vals) {
    geom_t g = {N, Na, Nd, S, R, ds};
    if (!geom_ok(&g)) return -1;
    const double h = 0.5 * (N - 1), hd = 0.5 * (Nd - 1);
    long nnz = 0;
    for (long ray = 0; ray < (long)Na * Nd; ++ray) {
        const int a = (int)(ray / Nd), d = (int)(ray % Nd);
        double c, s;
        int rd;
        angle(&g, a, &c, &s, &rd);
        const double sd = (d - hd) * ds;
        const double scale = 1.0 / fabs(rd ? c : s);
        for (int t = 0; t < N; ++t) {
            const double u = rd ? (sd - (t - h) * s) / c + h : (sd - (t - h) * c) / s + h;
            const double fl = floor(u);
            const long k0 = (long)fl;
            const double f = u - fl;
            for (int e = 0; e < 2; ++e) {
                const long k = k0 + e;
                const double w = (e ? f : 1.0 - f) * scale;
                if (k < 0 || k >= N || w == 0.0) continue;
                rows[nnz] = ray;
                cols[nnz] = rd ? (long)t * N + k : k * N + t;
                vals[nnz] = w;
                ++nnz;
            }
        }
    }
    return nnz;
}

/* Explicit B as (row = pixel, col = ray, val) triplets.
 * Capacity needed: 2 * N * N * N_a.  Returns the count, or -1. */
long orc_backproject_triplets(int N, int Na, int Nd, double S, double R, double ds,
                              int64_t *rows, int64_t *cols, double *vals) {
    geom_t g = {N, Na, Nd, S, R, ds};
    if (!geom_ok(&g)) return -1;
    const double h = 0.5 * (N - 1), hd = 0.5 * (Nd - 1);
    long nnz = 0;
    for (long p = 0; p < (long)N * N; ++p) {
        const int i = (int)(p / N), j = (int)(p % N);
        for (int a = 0; a < Na; ++a) {
            double c, s;
            int rd;
            angle(&g, a, &c, &s, &rd);
            const double u = ((j - h) * c + (i - h) * s) / ds + hd;
            const double fl = floor(u);
            const long d0 = (long)fl;
            const double f = u - fl;
            for (int e = 0; e < 2; ++e) {
                const long d = d0 + e;
                const double w = e ? f : 1.0 - f;
                if (d < 0 || d >= Nd || w == 0.0) continue;
                rows[nnz] = p;
                cols[nnz] = (long)a * Nd + d;
                vals[nnz] = w;
                ++nnz;
            }
        }
    }
    return nnz;
}
