/*
 * nif_oracle.c -- plain FP64 CPU oracle for the geometric stages of the
 * voxel deformation-aware neural intersection function.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library. The product path (the
 * CUDA library and its Python binding) never calls it and shares no code
 * with it.
 *
 * Everything here is written for clarity, not speed: brute force over every
 * occupied voxel and every triangle, in double precision, with OpenMP over
 * rays only so that the CPU baseline uses the host's cores.
 *
 * Contents (paper section each function follows):
 *   - parameterized deformation and its inverse (Sec. 2: the rest space and
 *     deformed space; the family bend o twist o taper is our reading, the
 *     paper names none),
 *   - rest-space voxelization of the mesh (Sec. 2),
 *   - ray / deformed-voxel segment lists (Sec. 2.1 and Sec. 2.2), defined as
 *     the hits of each occupied voxel's triangulated deformed hull, or of its
 *     six faces taken as bilinear patches (the paper fixes neither),
 *   - ground-truth labels of the locally linearized rest-space segment
 *     (Sec. 2: "intersect the locally linearized rays with the rest-space
 *     geometry"),
 *   - exact deformed-space ray / deformed-mesh intersection (the ground
 *     truth the approximation is judged against).
 *
 * Compile with -ffp-contract=off: the voxelization decision is made in
 * IEEE double without fused multiply-add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_CX 0.5
#define OR_CY 0.5
#define OR_CZ 0.5
/* bend parameter b in [-1,1] is the curvature kappa = OR_KBEND * b */
#define OR_KBEND 0.75

/* ------------------------------------------------------------------------ */
/* Deformation D = Bend o Twist o Taper about the cube centre c.             */
/* ------------------------------------------------------------------------ */

/* sin(u)/u and the two bend helper ratios, with their Taylor series near 0 */
static double sinc_(double u) { return fabs(u) < 1e-4 ? 1.0 - u * u / 6.0 : sin(u) / u; }
static double atanc_(double u) { return fabs(u) < 1e-4 ? 1.0 - u * u / 3.0 : atan(u) / u; }

/* Taper: s = 1 + a*z, (x, y, z) -> (s x, s y, z). */
static void taper_fwd(double a, const double p[3], double q[3]) {
    double s = 1.0 + a * p[2];
    q[0] = s * p[0]; q[1] = s * p[1]; q[2] = p[2];
}
static void taper_inv(double a, const double q[3], double p[3]) {
    double s = 1.0 + a * q[2];
    p[0] = q[0] / s; p[1] = q[1] / s; p[2] = q[2];
}
/* Twist about z: rotate (x, y) by alpha = theta*z. */
static void twist_fwd(double th, const double p[3], double q[3]) {
    double al = th * p[2], c = cos(al), s = sin(al);
    q[0] = c * p[0] - s * p[1]; q[1] = s * p[0] + c * p[1]; q[2] = p[2];
}
static void twist_inv(double th, const double q[3], double p[3]) {
    double al = th * q[2], c = cos(al), s = sin(al);
    p[0] = c * q[0] + s * q[1]; p[1] = -s * q[0] + c * q[1]; p[2] = q[2];
}
/* Bend in the x-z plane about an axis parallel to y (Barr 1984), curvature
 * k, bend angle beta = k*z:  X = R - (R - x) cos(beta), Z = (R - x) sin(beta)
 * with R = 1/k, written without 1/k so that k -> 0 is the identity:
 *   X = x cos(beta) + z sin(beta/2) sinc(beta/2),  Z = z sinc(beta) - x sin(beta). */
static void bend_fwd(double k, const double p[3], double q[3]) {
    double b = k * p[2];
    double h = 0.5 * b;
    q[0] = p[0] * cos(b) + p[2] * sin(h) * sinc_(h);
    q[1] = p[1];
    q[2] = p[2] * sinc_(b) - p[0] * sin(b);
}
/* Inverse bend: with g = 1 - k X and the bend angle beta = atan(k Z / g),
 *   x = (2X - k (X^2 + Z^2)) / (1 + sqrt(g^2 + (k Z)^2)),  z = (Z / g) atanc(k Z / g). */
static void bend_inv(double k, const double q[3], double p[3]) {
    double X = q[0], Z = q[2];
    double g = 1.0 - k * X, hz = k * Z;
    double r = sqrt(g * g + hz * hz);
    p[0] = (2.0 * X - k * (X * X + Z * Z)) / (1.0 + r);
    p[1] = q[1];
    p[2] = (Z / g) * atanc_(hz / g);
}

/* pose = (bend, twist, taper) */
void or_deform(const double* pose, const double* x, double* y, long n) {
    double k = OR_KBEND * pose[0];
    for (long i = 0; i < n; i++) {
        double p[3] = {x[3 * i] - OR_CX, x[3 * i + 1] - OR_CY, x[3 * i + 2] - OR_CZ};
        double a[3], b[3], c[3];
        taper_fwd(pose[2], p, a);
        twist_fwd(pose[1], a, b);
        bend_fwd(k, b, c);
        y[3 * i] = c[0] + OR_CX; y[3 * i + 1] = c[1] + OR_CY; y[3 * i + 2] = c[2] + OR_CZ;
    }
}

void or_inverse(const double* pose, const double* y, double* x, long n) {
    double k = OR_KBEND * pose[0];
    for (long i = 0; i < n; i++) {
        double q[3] = {y[3 * i] - OR_CX, y[3 * i + 1] - OR_CY, y[3 * i + 2] - OR_CZ};
        double a[3], b[3], c[3];
        bend_inv(k, q, a);
        twist_inv(pose[1], a, b);
        taper_inv(pose[2], b, c);
        x[3 * i] = c[0] + OR_CX; x[3 * i + 1] = c[1] + OR_CY; x[3 * i + 2] = c[2] + OR_CZ;
    }
}

static void matmul3(const double A[9], const double B[9], double C[9]) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    memcpy(C, T, sizeof T);
}

/* Jacobians of the three stages (row-major 3x3) and of the parameters.
 *   J      = dD/dx at the rest point x        (J[3*i+j] = dy_i/dx_j)
 *   Jp     = dD/d(bend, twist, taper) at x     (Jp[3*i+j] = dy_i/dparam_j)   */
void or_jacobians(const double* pose, const double* x, double* J, double* Jp, long n) {
    double k = OR_KBEND * pose[0], th = pose[1], ta = pose[2];
    for (long i = 0; i < n; i++) {
        double p[3] = {x[3 * i] - OR_CX, x[3 * i + 1] - OR_CY, x[3 * i + 2] - OR_CZ};
        double p1[3], p2[3];
        taper_fwd(ta, p, p1);
        twist_fwd(th, p1, p2);
        double s = 1.0 + ta * p[2];
        double Jt[9] = {s, 0, ta * p[0], 0, s, ta * p[1], 0, 0, 1};
        double al = th * p1[2], ca = cos(al), sa = sin(al);
        double Jw[9] = {ca, -sa, -th * p2[1], sa, ca, th * p2[0], 0, 0, 1};
        double be = k * p2[2], cb = cos(be), sb = sin(be), m = 1.0 - k * p2[0];
        double Jb[9] = {cb, 0, m * sb, 0, 1, 0, -sb, 0, m * cb};
        double T[9];
        matmul3(Jb, Jw, T);
        matmul3(T, Jt, J + 9 * i);
        /* parameter derivatives */
        double dp1_dta[3] = {p[2] * p[0], p[2] * p[1], 0};
        double dp2_dth[3] = {-p2[2] * p2[1], p2[2] * p2[0], 0};
        /* d(bend)/dk at fixed (x, z) = p2, with beta = k z:
         *   dX/dk = -x z sin(beta) + z^2 (beta sin(beta) - 1 + cos(beta)) / beta^2
         *   dZ/dk = -x z cos(beta) + z^2 (beta cos(beta) - sin(beta)) / beta^2     */
        double z = p2[2], xx = p2[0];
        double h1, h2;
        if (fabs(be) < 1e-3) {
            h1 = 0.5 - be * be / 8.0;
            h2 = -be / 3.0 + be * be * be / 30.0;
        } else {
            h1 = (be * sb - 1.0 + cb) / (be * be);
            h2 = (be * cb - sb) / (be * be);
        }
        double dk[3] = {-xx * z * sb + z * z * h1, 0, -xx * z * cb + z * z * h2};
        double a1[3], a2[3];
        for (int r = 0; r < 3; r++) a1[r] = Jw[3 * r] * dp1_dta[0] + Jw[3 * r + 1] * dp1_dta[1] + Jw[3 * r + 2] * dp1_dta[2];
        for (int r = 0; r < 3; r++) a2[r] = Jb[3 * r] * a1[0] + Jb[3 * r + 1] * a1[1] + Jb[3 * r + 2] * a1[2];
        double b2[3];
        for (int r = 0; r < 3; r++) b2[r] = Jb[3 * r] * dp2_dth[0] + Jb[3 * r + 1] * dp2_dth[1] + Jb[3 * r + 2] * dp2_dth[2];
        double* P = Jp + 9 * i;
        for (int r = 0; r < 3; r++) {
            P[3 * r + 0] = OR_KBEND * dk[r];
            P[3 * r + 1] = b2[r];
            P[3 * r + 2] = a2[r];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Rest-space voxelization: triangle / box overlap by the separating axis    */
/* theorem (Akenine-Moeller 2001), voxel boxes dilated by OR_EPSV.           */
/* ------------------------------------------------------------------------ */
#define OR_EPSV 1e-7

static int plane_box(const double n[3], const double v[3], double h) {
    double vmin[3], vmax[3];
    for (int q = 0; q < 3; q++) {
        if (n[q] > 0.0) { vmin[q] = -h - v[q]; vmax[q] = h - v[q]; }
        else            { vmin[q] = h - v[q];  vmax[q] = -h - v[q]; }
    }
    double dmin = n[0] * vmin[0] + n[1] * vmin[1] + n[2] * vmin[2];
    double dmax = n[0] * vmax[0] + n[1] * vmax[1] + n[2] * vmax[2];
    if (dmin > 0.0) return 0;
    if (dmax >= 0.0) return 1;
    return 0;
}

/* Triangle (v0,v1,v2) vs cube of half-size h centred at c. */
static int tri_box(const double c[3], double h, const double* a, const double* b, const double* d) {
    double v0[3], v1[3], v2[3], e0[3], e1[3], e2[3];
    for (int q = 0; q < 3; q++) { v0[q] = a[q] - c[q]; v1[q] = b[q] - c[q]; v2[q] = d[q] - c[q]; }
    for (int q = 0; q < 3; q++) { e0[q] = v1[q] - v0[q]; e1[q] = v2[q] - v1[q]; e2[q] = v0[q] - v2[q]; }
    const double* E[3] = {e0, e1, e2};
    const double* V[3] = {v0, v1, v2};
    /* 9 cross-product axes: e_i x X, e_i x Y, e_i x Z */
    for (int i = 0; i < 3; i++) {
        const double* e = E[i];
        /* the two vertices not on edge i's start give distinct projections; all three are tested */
        for (int ax = 0; ax < 3; ax++) {
            double p[3];
            double rad;
            int u = (ax + 1) % 3, w = (ax + 2) % 3;
            /* axis = e x unit(ax): components along u and w are (e[w], -e[u]) up to ordering */
            for (int k = 0; k < 3; k++) p[k] = e[w] * V[k][u] - e[u] * V[k][w];
            rad = (fabs(e[w]) + fabs(e[u])) * h;
            double mn = p[0], mx = p[0];
            for (int k = 1; k < 3; k++) { if (p[k] < mn) mn = p[k]; if (p[k] > mx) mx = p[k]; }
            if (mn > rad || mx < -rad) return 0;
        }
    }
    /* 3 box face normals */
    for (int q = 0; q < 3; q++) {
        double mn = v0[q], mx = v0[q];
        if (v1[q] < mn) mn = v1[q];
        if (v1[q] > mx) mx = v1[q];
        if (v2[q] < mn) mn = v2[q];
        if (v2[q] > mx) mx = v2[q];
        if (mn > h || mx < -h) return 0;
    }
    /* triangle plane */
    double n[3] = {e0[1] * e1[2] - e0[2] * e1[1], e0[2] * e1[0] - e0[0] * e1[2], e0[0] * e1[1] - e0[1] * e1[0]};
    return plane_box(n, v0, h);
}

/* occ[N^3] (x fastest) = 1 if some triangle overlaps the dilated voxel box.
 * If tri_ptr != NULL, also fills the CSR of triangles per voxel (all N^3
 * voxels, ascending triangle id) up to `cap` entries; returns the total
 * number of (voxel, triangle) pairs. */
long or_voxelize(int N, const float* verts, const int* tris, int nt, uint8_t* occ,
                 long* tri_ptr, int* tri_idx, long cap) {
    long nvox = (long)N * N * N;
    memset(occ, 0, (size_t)nvox);
    int* cnt = (int*)calloc((size_t)nvox, sizeof(int));
    double h = 0.5 / N + OR_EPSV;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            if (!tri_ptr) break;
            tri_ptr[0] = 0;
            for (long v = 0; v < nvox; v++) tri_ptr[v + 1] = tri_ptr[v] + cnt[v];
            memset(cnt, 0, (size_t)nvox * sizeof(int));
        }
        for (int t = 0; t < nt; t++) {
            double P[3][3];
            double lo[3] = {1e30, 1e30, 1e30}, hi[3] = {-1e30, -1e30, -1e30};
            for (int k = 0; k < 3; k++)
                for (int q = 0; q < 3; q++) {
                    P[k][q] = (double)verts[3 * tris[3 * t + k] + q];
                    if (P[k][q] < lo[q]) lo[q] = P[k][q];
                    if (P[k][q] > hi[q]) hi[q] = P[k][q];
                }
            int i0[3], i1[3];
            for (int q = 0; q < 3; q++) {
                i0[q] = (int)floor((lo[q] - 2 * OR_EPSV) * N) - 1;
                i1[q] = (int)floor((hi[q] + 2 * OR_EPSV) * N) + 1;
                if (i0[q] < 0) i0[q] = 0;
                if (i1[q] > N - 1) i1[q] = N - 1;
            }
            for (int k = i0[2]; k <= i1[2]; k++)
                for (int j = i0[1]; j <= i1[1]; j++)
                    for (int i = i0[0]; i <= i1[0]; i++) {
                        double c[3] = {(i + 0.5) / N, (j + 0.5) / N, (k + 0.5) / N};
                        if (!tri_box(c, h, P[0], P[1], P[2])) continue;
                        long v = i + (long)N * (j + (long)N * k);
                        if (pass == 0) { occ[v] = 1; cnt[v]++; }
                        else {
                            long pos = tri_ptr[v] + cnt[v]++;
                            if (pos < cap) tri_idx[pos] = t;
                        }
                    }
        }
    }
    long total = 0;
    for (long v = 0; v < nvox; v++) total += cnt[v];
    free(cnt);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Ray / deformed voxel hull.                                                */
/* The hull of voxel (i,j,k) is the hexahedron whose corners are the         */
/* deformed lattice points D((i+a)/N, (j+b)/N, (k+c)/N), a,b,c in {0,1}.     */
/* Each face is split into two triangles along the diagonal that starts at   */
/* the face corner of smallest lattice index.                                */
/* ------------------------------------------------------------------------ */

/* Faces as local corner ids (bit0 = a, bit1 = b, bit2 = c): lowest corner,
 * the two side corners, highest corner. Triangles: (lo,s1,hi), (lo,s2,hi). */
static const int OR_FACES[6][4] = {
    {0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};

/* Moeller-Trumbore, double, two-sided. Returns 1 on a hit of the plane
 * inside the closed triangle; t along the (not necessarily unit) direction. */
static int mt_hit(const double o[3], const double d[3], const double* A, const double* B,
                  const double* C, double* t, double* u, double* v) {
    double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
    double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
    if (det == 0.0) { *t = 1e300; *u = -1.0; *v = -1.0; return 0; }
    double inv = 1.0 / det;
    double s[3] = {o[0] - A[0], o[1] - A[1], o[2] - A[2]};
    double uu = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
    double q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
    double vv = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * inv;
    double tt = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * inv;
    *t = tt; *u = uu; *v = vv;
    return (uu >= 0.0 && vv >= 0.0 && uu + vv <= 1.0);
}

/* distance between the line o + t d (all t) and the segment [A,B] */
static double line_seg_dist(const double o[3], const double d[3], const double* A, const double* B) {
    double e[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double w[3] = {A[0] - o[0], A[1] - o[1], A[2] - o[2]};
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    double de = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
    double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
    double ew = e[0] * w[0] + e[1] * w[1] + e[2] * w[2];
    double den = dd * ee - de * de;
    double s; /* parameter on segment */
    if (den <= 1e-300) s = 0.0;
    else s = (de * dw - dd * ew) / den;
    if (s < 0.0) s = 0.0;
    if (s > 1.0) s = 1.0;
    double P[3] = {A[0] + s * e[0], A[1] + s * e[1], A[2] + s * e[2]};
    double tt = ((P[0] - o[0]) * d[0] + (P[1] - o[1]) * d[1] + (P[2] - o[2]) * d[2]) / dd;
    double Q[3] = {o[0] + tt * d[0] - P[0], o[1] + tt * d[1] - P[1], o[2] + tt * d[2] - P[2]};
    return sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2]);
}

/* distance from the point X to the segment [A,B] */
static double point_seg_dist(const double X[3], const double* A, const double* B) {
    double e[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double w[3] = {X[0] - A[0], X[1] - A[1], X[2] - A[2]};
    double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    double s = ee > 0 ? (e[0] * w[0] + e[1] * w[1] + e[2] * w[2]) / ee : 0.0;
    if (s < 0.0) s = 0.0;
    if (s > 1.0) s = 1.0;
    double q[3] = {w[0] - s * e[0], w[1] - s * e[1], w[2] - s * e[2]};
    return sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
}

/* Deformed corners of voxel (i,j,k): X[8][3], local id = a + 2b + 4c. With
 * `lattice` (deformed positions of all (N+1)^3 lattice corners, index
 * a + (N+1)(b + (N+1)c), as a learned deformation field gives them) the
 * corners are read from it instead of deforming by the pose. */
static void hull_corners(int N, int i, int j, int k, const double* pose, const double* lattice, double X[8][3]) {
    if (lattice) {
        const long M = N + 1;
        for (int c = 0; c < 8; c++) {
            const long a = i + (c & 1), b = j + ((c >> 1) & 1), e = k + ((c >> 2) & 1);
            const double* L = lattice + 3 * (a + M * (b + M * e));
            X[c][0] = L[0];
            X[c][1] = L[1];
            X[c][2] = L[2];
        }
        return;
    }
    double P[24];
    for (int c = 0; c < 8; c++) {
        P[3 * c + 0] = (double)(i + (c & 1)) / N;
        P[3 * c + 1] = (double)(j + ((c >> 1) & 1)) / N;
        P[3 * c + 2] = (double)(k + ((c >> 2) & 1)) / N;
    }
    or_deform(pose, P, &X[0][0], 8);
}

/*
 * Line / bilinear patch (the curved-face reading of a deformed voxel): the
 * face with corners P00, P10, P01, P11 is the surface
 *   S(u,v) = P00 + u (P10 - P00) + v (P01 - P00) + u v (P11 - P10 - P01 + P00),
 * u, v in [0,1]. Points of the line o + t d are exactly those whose
 * components along two vectors n1, n2 orthogonal to d (and to each other)
 * vanish after subtracting o, so a hit solves the pair of scalar bilinear
 * equations x(u,v) = y(u,v) = 0 of the projected corners. Eliminating v
 * gives a quadratic in u: with h, e, f, g the projected P00 - o, P10 - P00,
 * P01 - P00 and P11 - P10 - P01 + P00 and k(a,b) = a_x b_y - a_y b_x,
 *   k(e,g) u^2 + (k(h,g) + k(e,f)) u + k(h,f) = 0,
 * and v follows from h + u e + v (f + u g) = 0. Returns the hits (0..2) with
 * u, v in [0,1]; t[i] along d (d of any length), sep = the distance between
 * the two roots' points when both are hits, else 1e300.
 */
int or_bilinear_hits(const double o[3], const double d[3], const double* P00, const double* P10,
                     const double* P01, const double* P11, double t[2], double uv[4], double* sep) {
    *sep = 1e300;
    /* n1 = d x (axis of the smallest |d| component), n2 = d x n1 */
    int ax = fabs(d[0]) <= fabs(d[1]) ? (fabs(d[0]) <= fabs(d[2]) ? 0 : 2) : (fabs(d[1]) <= fabs(d[2]) ? 1 : 2);
    double a[3] = {0.0, 0.0, 0.0};
    a[ax] = 1.0;
    double n1[3] = {d[1] * a[2] - d[2] * a[1], d[2] * a[0] - d[0] * a[2], d[0] * a[1] - d[1] * a[0]};
    double n2[3] = {d[1] * n1[2] - d[2] * n1[1], d[2] * n1[0] - d[0] * n1[2], d[0] * n1[1] - d[1] * n1[0]};
    const double* P[4] = {P00, P10, P01, P11};
    double X[4], Y[4];
    for (int c = 0; c < 4; c++) {
        double w[3] = {P[c][0] - o[0], P[c][1] - o[1], P[c][2] - o[2]};
        X[c] = n1[0] * w[0] + n1[1] * w[1] + n1[2] * w[2];
        Y[c] = n2[0] * w[0] + n2[1] * w[1] + n2[2] * w[2];
    }
    double h[2] = {X[0], Y[0]};
    double e[2] = {X[1] - X[0], Y[1] - Y[0]};
    double f[2] = {X[2] - X[0], Y[2] - Y[0]};
    double g[2] = {X[3] - X[2] - X[1] + X[0], Y[3] - Y[2] - Y[1] + Y[0]};
#define OR_K(p, q) ((p)[0] * (q)[1] - (p)[1] * (q)[0])
    double k2 = OR_K(e, g), k1 = OR_K(h, g) + OR_K(e, f), k0 = OR_K(h, f);
#undef OR_K
    double us[2];
    int nu = 0;
    double scale = fabs(k2) + fabs(k1) + fabs(k0);
    if (scale == 0.0) return 0;
    if (fabs(k2) <= 1e-14 * scale) {
        if (k1 != 0.0) us[nu++] = -k0 / k1;
    } else {
        double disc = k1 * k1 - 4.0 * k2 * k0;
        if (disc < 0.0) return 0;
        double sq = sqrt(disc);
        double q = -0.5 * (k1 + (k1 >= 0.0 ? sq : -sq));
        us[nu++] = q / k2;
        if (disc > 0.0 && q != 0.0) us[nu++] = k0 / q;
    }
    int n = 0;
    double pts[2][3];
    for (int i = 0; i < nu; i++) {
        double u = us[i];
        if (!(u >= 0.0 && u <= 1.0)) continue;
        double w[2] = {f[0] + u * g[0], f[1] + u * g[1]};
        double r[2] = {h[0] + u * e[0], h[1] + u * e[1]};
        double ww = w[0] * w[0] + w[1] * w[1];
        if (ww == 0.0) continue;
        double v = -(r[0] * w[0] + r[1] * w[1]) / ww;
        if (!(v >= 0.0 && v <= 1.0)) continue;
        double S[3];
        for (int k = 0; k < 3; k++)
            S[k] = P00[k] + u * (P10[k] - P00[k]) + v * (P01[k] - P00[k]) + u * v * (P11[k] - P10[k] - P01[k] + P00[k]);
        double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        t[n] = ((S[0] - o[0]) * d[0] + (S[1] - o[1]) * d[1] + (S[2] - o[2]) * d[2]) / dd;
        uv[2 * n] = u;
        uv[2 * n + 1] = v;
        for (int k = 0; k < 3; k++) pts[n][k] = S[k];
        n++;
    }
    if (n == 2) {
        double q[3] = {pts[1][0] - pts[0][0], pts[1][1] - pts[0][1], pts[1][2] - pts[0][2]};
        *sep = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    }
    return n;
}

typedef struct { int v; double t0, t1; } or_seg;

static int seg_cmp(const void* a, const void* b) {
    const or_seg* x = (const or_seg*)a;
    const or_seg* y = (const or_seg*)b;
    if (x->t0 < y->t0) return -1;
    if (x->t0 > y->t0) return 1;
    return (x->v > y->v) - (x->v < y->v);
}

/*
 * Segment list of every ray (Sec. 2.1, Sec. 2.2): for each occupied voxel v,
 * all hits of the ray line with the 12 hull triangles (bilinear = 0) or with
 * the 6 bilinear face patches (bilinear = 1, faces as corner quads
 * (lo, s1, s2, hi) = (P00, P10, P01, P11)); with at least two hits,
 * t0 = max(min t, tmin), t1 = min(max t, tmax); a segment exists when
 * t1 > t0. Segments are sorted by (t0, v).
 *
 * rays: float [n, 8] = o, d, tmin, tmax. Outputs per ray: count[r], and
 * vox/t0/t1 at [r*max_per_ray + s]. margin[r] = the smallest decision margin
 * met by the ray (world units): the length of any segment, the distance of
 * the ray to any occupied hull it misses, the gap between consecutive t0.
 * Returns the number of rays that overflowed max_per_ray.
 */
long or_segments(int N, const uint8_t* occ, const double* pose, const float* rays, long n,
                 int max_per_ray, int* count, int* vox, double* t0, double* t1, double* margin, int bilinear,
                 const double* lattice) {
    long nvox = (long)N * N * N;
    long nocc = 0;
    for (long v = 0; v < nvox; v++) nocc += occ[v] != 0;
    int* list = (int*)malloc(sizeof(int) * (size_t)(nocc ? nocc : 1));
    nocc = 0;
    for (long v = 0; v < nvox; v++) if (occ[v]) list[nocc++] = (int)v;
    /* deformed corners of every occupied voxel, once */
    double (*X)[8][3] = (double (*)[8][3])malloc(sizeof(double) * 24 * (size_t)(nocc ? nocc : 1));
    double (*bmin)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(nocc ? nocc : 1));
    double (*bmax)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (size_t)(nocc ? nocc : 1));
    for (long q = 0; q < nocc; q++) {
        int v = list[q];
        hull_corners(N, v % N, (v / N) % N, v / (N * N), pose, lattice, X[q]);
        for (int a = 0; a < 3; a++) { bmin[q][a] = 1e300; bmax[q][a] = -1e300; }
        for (int c = 0; c < 8; c++)
            for (int a = 0; a < 3; a++) {
                if (X[q][c][a] < bmin[q][a]) bmin[q][a] = X[q][c][a];
                if (X[q][c][a] > bmax[q][a]) bmax[q][a] = X[q][c][a];
            }
    }
    long overflow = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : overflow)
    for (long r = 0; r < n; r++) {
        const float* R = rays + 8 * r;
        double o[3] = {R[0], R[1], R[2]}, d[3] = {R[3], R[4], R[5]};
        double tmin = R[6], tmax = R[7];
        or_seg* segs = (or_seg*)malloc(sizeof(or_seg) * (size_t)(max_per_ray + 1));
        int ns = 0;
        double mar = 1e300;
        for (long q = 0; q < nocc; q++) {
            double tlo = 1e300, thi = -1e300;
            int hits = 0;
            for (int f = 0; f < 6; f++) {
                const int* F = OR_FACES[f];
                if (bilinear) {
                    double tt[2], uv[4], sep;
                    int k = or_bilinear_hits(o, d, X[q][F[0]], X[q][F[1]], X[q][F[2]], X[q][F[3]], tt, uv, &sep);
                    for (int i = 0; i < k; i++) {
                        hits++;
                        if (tt[i] < tlo) tlo = tt[i];
                        if (tt[i] > thi) thi = tt[i];
                    }
                    if (sep < mar) mar = sep;      /* a near-tangent pair of hits */
                    continue;
                }
                for (int s = 1; s <= 2; s++) {
                    double t, u, w;
                    if (mt_hit(o, d, X[q][F[0]], X[q][F[s]], X[q][F[3]], &t, &u, &w)) {
                        hits++;
                        if (t < tlo) tlo = t;
                        if (t > thi) thi = t;
                    }
                }
            }
            int made = 0;
            if (hits >= 2) {
                double a = tlo > tmin ? tlo : tmin, b = thi < tmax ? thi : tmax;
                if (b > a) {
                    made = 1;
                    if (b - a < mar) mar = b - a;
                    if (ns < max_per_ray) { segs[ns].v = list[q]; segs[ns].t0 = a; segs[ns].t1 = b; }
                    ns++;
                }
            }
            if (!made || bilinear) {
                /* near miss? distance to the hull's edges if the ray meets the slightly grown box
                 * (curved faces: for hit hulls too, since a hit next to a face edge is not
                 * decided identically from the two faces that share it in finite precision) */
                double g = 1e-3, ta = -1e300, tb = 1e300;
                for (int a = 0; a < 3; a++) {
                    double lo = bmin[q][a] - g, hi = bmax[q][a] + g;
                    if (d[a] == 0.0) { if (o[a] < lo || o[a] > hi) { ta = 1; tb = 0; } continue; }
                    double u0 = (lo - o[a]) / d[a], u1 = (hi - o[a]) / d[a];
                    if (u0 > u1) { double tt = u0; u0 = u1; u1 = tt; }
                    if (u0 > ta) ta = u0;
                    if (u1 < tb) tb = u1;
                }
                if (ta <= tb) {
                    for (int f = 0; f < 6; f++) {
                        const int* F = OR_FACES[f];
                        const int ed[5][2] = {{F[0], F[1]}, {F[1], F[3]}, {F[3], F[2]}, {F[2], F[0]}, {F[0], F[3]}};
                        for (int e = 0; e < 5; e++) {
                            double dist = line_seg_dist(o, d, X[q][ed[e][0]], X[q][ed[e][1]]);
                            if (dist < mar) mar = dist;
                        }
                    }
                }
            }
        }
        if (ns > max_per_ray) { overflow++; ns = max_per_ray; }
        qsort(segs, (size_t)ns, sizeof(or_seg), seg_cmp);
        for (int s = 1; s < ns; s++) {
            double g = segs[s].t0 - segs[s - 1].t0;
            if (g < mar) mar = g;
        }
        count[r] = ns;
        for (int s = 0; s < ns; s++) {
            vox[r * (long)max_per_ray + s] = segs[s].v;
            t0[r * (long)max_per_ray + s] = segs[s].t0;
            t1[r * (long)max_per_ray + s] = segs[s].t1;
        }
        margin[r] = mar;
        free(segs);
    }
    free(list); free(X); free(bmin); free(bmax);
    return overflow;
}

/* ------------------------------------------------------------------------ */
/* Ground-truth labels of a linearized rest-space segment (Sec. 2).          */
/* ------------------------------------------------------------------------ */

/*
 * For each segment s: the straight rest segment p0[s] -> p1[s] is intersected
 * with the triangles listed for its voxel vox[s]; the label is the first hit
 * (smallest parameter in [0,1], ties to the smaller triangle id).
 * Outputs: occ[s] (0/1), tpar[s] (parameter in [0,1] of the hit), normal
 * (unit geometric normal of the hit triangle, from its winding), albedo,
 * material, and margin[s]: the smallest distance (world units) from the
 * segment's line crossing of any listed triangle's plane to that triangle's
 * edges, of a hit to the segment's ends, or between two hits.
 */
void or_labels(const long* tri_ptr, const int* tri_idx, const float* verts, const int* tris,
               const float* tri_albedo, const uint8_t* tri_mat, long nseg, const int* vox,
               const double* p0, const double* p1, uint8_t* occ, double* tpar, double* normal,
               double* albedo, uint8_t* mat, double* margin) {
#pragma omp parallel for schedule(dynamic, 256)
    for (long s = 0; s < nseg; s++) {
        const double* a = p0 + 3 * s;
        double d[3] = {p1[3 * s] - a[0], p1[3 * s + 1] - a[1], p1[3 * s + 2] - a[2]};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double best = 1e300, second = 1e300, mar = 1e300;
        int bt = -1;
        for (long q = tri_ptr[vox[s]]; q < tri_ptr[vox[s] + 1]; q++) {
            int t = tri_idx[q];
            double P[3][3];
            for (int k = 0; k < 3; k++)
                for (int c = 0; c < 3; c++) P[k][c] = verts[3 * tris[3 * t + k] + c];
            double tt, u, v;
            int in = mt_hit(a, d, P[0], P[1], P[2], &tt, &u, &v);
            /* plane crossing near the segment: distance to the triangle's boundary */
            if (tt > -0.5 && tt < 1.5) {
                double w = 1.0 - u - v;
                double X[3];
                for (int c = 0; c < 3; c++) X[c] = a[c] + tt * d[c];
                double db;
                if (in) {
                    double e[3][3];
                    for (int c = 0; c < 3; c++) {
                        e[0][c] = P[1][c] - P[0][c]; e[1][c] = P[2][c] - P[1][c]; e[2][c] = P[0][c] - P[2][c];
                    }
                    double nrm[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                                     e[0][0] * e[1][1] - e[0][1] * e[1][0]};
                    double area2 = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
                    double L0 = sqrt(e[1][0] * e[1][0] + e[1][1] * e[1][1] + e[1][2] * e[1][2]);
                    double L1 = sqrt(e[2][0] * e[2][0] + e[2][1] * e[2][1] + e[2][2] * e[2][2]);
                    double L2 = sqrt(e[0][0] * e[0][0] + e[0][1] * e[0][1] + e[0][2] * e[0][2]);
                    /* barycentric (w at P0, u at P1, v at P2) times the altitude to the opposite edge */
                    double m0 = fabs(w) * area2 / L0, m1 = fabs(u) * area2 / L1, m2 = fabs(v) * area2 / L2;
                    db = m0 < m1 ? m0 : m1;
                    if (m2 < db) db = m2;
                } else {
                    double d0 = point_seg_dist(X, P[0], P[1]), d1 = point_seg_dist(X, P[1], P[2]);
                    double d2 = point_seg_dist(X, P[2], P[0]);
                    db = d0 < d1 ? d0 : d1;
                    if (d2 < db) db = d2;
                }
                if (tt >= 0.0 && tt <= 1.0 && db < mar) mar = db;
                if (in) {
                    double dt = fabs(tt) * len, dt1 = fabs(1.0 - tt) * len;
                    if (dt < mar) mar = dt;
                    if (dt1 < mar) mar = dt1;
                }
            }
            if (in && tt >= 0.0 && tt <= 1.0) {
                if (tt < best || (tt == best && t < bt)) { second = best; best = tt; bt = t; }
                else if (tt < second) second = tt;
            }
        }
        if (bt >= 0 && second < 1e300 && (second - best) * len < mar) mar = (second - best) * len;
        margin[s] = mar;
        if (bt < 0) {
            occ[s] = 0; tpar[s] = 0;
            for (int c = 0; c < 3; c++) { normal[3 * s + c] = 0; albedo[3 * s + c] = 0; }
            mat[s] = 0;
            continue;
        }
        occ[s] = 1; tpar[s] = best;
        double P[3][3];
        for (int k = 0; k < 3; k++)
            for (int c = 0; c < 3; c++) P[k][c] = verts[3 * tris[3 * bt + k] + c];
        double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
        double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
        double nrm[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        for (int c = 0; c < 3; c++) {
            normal[3 * s + c] = nrm[c] / nl;
            albedo[3 * s + c] = tri_albedo[3 * bt + c];
        }
        mat[s] = tri_mat[bt];
    }
}

/* ------------------------------------------------------------------------ */
/* Exact deformed-space ground truth: every ray against every triangle of    */
/* the deformed mesh (vertices already deformed, double).                    */
/* ------------------------------------------------------------------------ */
void or_exact_hits(const double* dverts, const int* tris, int nt, const float* rays, long n,
                   double* thit, int* tri_hit) {
#pragma omp parallel for schedule(dynamic, 16)
    for (long r = 0; r < n; r++) {
        const float* R = rays + 8 * r;
        double o[3] = {R[0], R[1], R[2]}, d[3] = {R[3], R[4], R[5]};
        double best = 1e300;
        int bt = -1;
        for (int t = 0; t < nt; t++) {
            double tt, u, v;
            if (mt_hit(o, d, dverts + 3 * tris[3 * t], dverts + 3 * tris[3 * t + 1],
                       dverts + 3 * tris[3 * t + 2], &tt, &u, &v)) {
                if (tt >= R[6] && tt <= R[7] && tt < best) { best = tt; bt = t; }
            }
        }
        thit[r] = bt >= 0 ? best : INFINITY;
        tri_hit[r] = bt;
    }
}

int or_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
