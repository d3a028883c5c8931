/*
 * hm_oracle.c -- CPU FP64 oracle for the hybrid mesh-Gaussian renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the renderer computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header or constant with the CUDA library.
 *
 * What it follows (arXiv 2506.06988):
 *   - Eq. 1: the Gaussian G(x) = exp(-1/2 (x-u)^T Sigma^-1 (x-u)).
 *   - Sec. 3.1: Sigma = R S S^T R^T and the projected covariance
 *     Sigma' = J W Sigma W^T J^T (affine Jacobian J of the projection).
 *   - Eq. 2: front-to-back alpha blending C(p) = sum_i c_i s_i prod_{j<i}(1-s_j),
 *     s_i = alpha_i G'_i(p).
 *   - Sec. 3.4 "Joint rasterization": only Gaussians in front of the mesh
 *     (D_gs < D_m) are blended; the mesh colour I_m (or the background I_bg
 *     where no triangle covers the pixel) is added weighted by the remaining
 *     transmittance T.
 *   - Sec. 3.1 "Textured mesh": barycentric interpolation of UVs and a texture
 *     lookup per pixel.
 *
 * Discretisation the paper leaves to the 3DGS code it builds on (Sec. 4.1);
 * each is a stated reading:
 *   - pixel (x,y) is sampled at its centre (x+1/2, y+1/2);
 *   - a Gaussian is a candidate for a pixel iff d^2 = D^T conic D <= 9 (its
 *     3-sigma ellipse), alpha = min(0.99, o G), skipped if alpha < 1/255,
 *     blending stops before a Gaussian that would drop T below 1e-4;
 *   - near plane z > 0.2 for Gaussians, 0.3 px^2 low-pass dilation of Sigma',
 *     the 1.3 x half-FOV clamp inside J, colour = max(0, 0.5 + SH);
 *   - mesh coverage: vertices projected in FP64, snapped to 1/256 px,
 *     exact integer edge functions with the top-left fill rule, two-sided;
 *     depth (Sec. 3.4 D_m): the view z of the snapped face at the pixel
 *     centre, evaluated in FP64 from the exact integer barycentric weights
 *     w_k and the vertices' 1/z_k (1/z is affine in screen space, so
 *     z = sum w_k / sum w_k (1/z_k)) and rounded once to FP32; the nearest
 *     FP32 depth wins, ties to the lower triangle index; perspective-correct
 *     UVs; bilinear clamp-to-edge texture fetch with texel centres at
 *     half-integers, row 0 at v = 0.
 *   - Gaussian depth key: z = R_2 . mean + t_2 evaluated in FP64 as
 *     fma(R20, x, fma(R21, y, fma(R22, z, t2))), rounded once to FP32.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared hm_oracle.c -lm
 * (-ffp-contract=off: every multiply-add below is exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* camera: c[0..8] = R row-major (world->camera), c[9..11] = t,              */
/*         c[12..15] = fx, fy, cx, cy                                        */
/* ------------------------------------------------------------------------ */

/* view-space coordinate k of world point p, FP64 with the fixed FMA order */
static double view_coord(const double *c, int k, double x, double y, double z) {
    return fma(c[3 * k + 0], x, fma(c[3 * k + 1], y, fma(c[3 * k + 2], z, c[9 + k])));
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================== */
/* Mesh rasterisation (Sec. 3.1 "Textured mesh", Sec. 3.4 I_m and D_m)       */
/* ======================================================================== */

typedef struct {
    int valid;
    int64_t X[3], Y[3];   /* snapped screen positions, in the face's vertex order */
    double iz[3];         /* 1 / view z per vertex */
    int ord[3];           /* vertex order with positive signed area */
    int64_t area2;        /* |signed double area| in (1/256 px)^2 */
    double pa, pb;        /* FP64 screen gradient of 1/z, per pixel (tolerance model only) */
} face_setup;

#define OR_SNAP 256.0
#define OR_GUARD 2097152.0 /* 2^21 px: faces reaching beyond are culled */

static void setup_face(const double *c, const double *verts, const int *f, double znear,
                       face_setup *s) {
    s->valid = 0;
    for (int k = 0; k < 3; k++) {
        const double *v = verts + 3 * (int64_t)f[k];
        double X = view_coord(c, 0, v[0], v[1], v[2]);
        double Y = view_coord(c, 1, v[0], v[1], v[2]);
        double Z = view_coord(c, 2, v[0], v[1], v[2]);
        if (!(Z > znear)) return;
        double sx = fma(c[12], X / Z, c[14]);
        double sy = fma(c[13], Y / Z, c[15]);
        if (!(fabs(sx) <= OR_GUARD && fabs(sy) <= OR_GUARD)) return;
        s->X[k] = llrint(sx * OR_SNAP);
        s->Y[k] = llrint(sy * OR_SNAP);
        s->iz[k] = 1.0 / Z;
    }
    int64_t e1x = s->X[1] - s->X[0], e1y = s->Y[1] - s->Y[0];
    int64_t e2x = s->X[2] - s->X[0], e2y = s->Y[2] - s->Y[0];
    int64_t a2 = e1x * e2y - e1y * e2x;
    if (a2 == 0) return;
    if (a2 > 0) { s->ord[0] = 0; s->ord[1] = 1; s->ord[2] = 2; s->area2 = a2; }
    else        { s->ord[0] = 0; s->ord[1] = 2; s->ord[2] = 1; s->area2 = -a2; }
    /* Screen gradient of 1/z (per pixel of offset from the face's first
     * vertex), FP64.  It does not enter the depth, which face_depth64 takes
     * from the barycentric weights; it only sizes the FP32 error band of a
     * rasteriser that evaluates the 1/z plane from that vertex (see
     * or_mesh_raster). */
    double d1 = s->iz[1] - s->iz[0], d2 = s->iz[2] - s->iz[0];
    s->pa = 256.0 * (d1 * (double)e2y - d2 * (double)e1y) / (double)a2;
    s->pb = 256.0 * (d2 * (double)e1x - d1 * (double)e2x) / (double)a2;
    s->valid = 1;
}

/* edge a->b of a positively oriented triangle (y down): inside has E > 0;
 * pixels exactly on an edge belong to it iff the edge is a top or left edge */
static int edge_covers(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py,
                       int64_t *E) {
    int64_t dx = bx - ax, dy = by - ay;
    int64_t e = dx * (py - ay) - dy * (px - ax);
    *E = e;
    if (e > 0) return 1;
    if (e < 0) return 0;
    return (dy < 0) || (dy == 0 && dx > 0);
}

/* Coverage of pixel centre (px,py) in 1/256 px; on success writes the
 * barycentric numerators w[k] for the face's vertex k (sum = area2). */
static int face_covers(const face_setup *s, int64_t px, int64_t py, int64_t w[3]) {
    const int *o = s->ord;
    int64_t e01, e12, e20;
    if (!edge_covers(s->X[o[0]], s->Y[o[0]], s->X[o[1]], s->Y[o[1]], px, py, &e01)) return 0;
    if (!edge_covers(s->X[o[1]], s->Y[o[1]], s->X[o[2]], s->Y[o[2]], px, py, &e12)) return 0;
    if (!edge_covers(s->X[o[2]], s->Y[o[2]], s->X[o[0]], s->Y[o[0]], px, py, &e20)) return 0;
    w[o[2]] = e01;  /* weight of a vertex = edge function of the opposite edge */
    w[o[0]] = e12;
    w[o[1]] = e20;
    return 1;
}

/* Sec. 3.4 D_m: view z of the snapped face at a covered centre, FP64.  With
 * w_k the exact integer edge-function weights (sum = area2), the screen-space
 * barycentrics are w_k / area2 and 1/z interpolates linearly in screen space,
 * so z = area2 / sum_k w_k (1/z_k). */
static double face_depth64(const face_setup *s, const int64_t w[3]) {
    double S = (double)w[0] * s->iz[0] + (double)w[1] * s->iz[1] + (double)w[2] * s->iz[2];
    return (double)s->area2 / S;
}

/* Relative FP32 error band of the depth at (px, py): a rasteriser that keeps
 * the 1/z plane as three FP32 coefficients anchored at the face's first
 * vertex and evaluates it with two FMAs and one reciprocal commits at most
 * (3 kappa + 3) u, u = 2^-24, with kappa = (|a U| + |b V| + |1/z_0|) / (1/z)
 * the condition number of that evaluation (coefficient and offset roundings,
 * two FMA roundings, the reciprocal, the FP32 rounding of this reference). */
static double face_depth_relband(const face_setup *s, int64_t px, int64_t py, double D64) {
    double U = (double)(px - s->X[0]) / 256.0, V = (double)(py - s->Y[0]) / 256.0;
    double kappa = (fabs(s->pa * U) + fabs(s->pb * V) + fabs(s->iz[0])) * D64;
    return (3.0 * kappa + 3.0) * 0x1p-24;
}

/* perspective-correct barycentrics (FP64) of a covered centre */
static double face_bary(const face_setup *s, const int64_t w[3], double b[3]) {
    double S = (double)w[0] * s->iz[0] + (double)w[1] * s->iz[1] + (double)w[2] * s->iz[2];
    for (int k = 0; k < 3; k++) b[k] = (double)w[k] * s->iz[k] / S;
    return S;
}

static double texel(const double *tex, int tw, int th, int x, int y, int ch) {
    if (x < 0) x = 0;
    if (x > tw - 1) x = tw - 1;
    if (y < 0) y = 0;
    if (y > th - 1) y = th - 1;
    return tex[((int64_t)y * tw + x) * 3 + ch];
}

/* bilinear, clamp-to-edge; texel (i,j) centred at ((i+1/2)/tw, (j+1/2)/th) */
static void sample_bilinear(const double *tex, int tw, int th, double u, double v, double out[3]) {
    double s = u * tw - 0.5, t = v * th - 0.5;
    double x0 = floor(s), y0 = floor(t);
    double fx = s - x0, fy = t - y0;
    int ix = (int)x0, iy = (int)y0;
    for (int ch = 0; ch < 3; ch++) {
        out[ch] = (1 - fx) * (1 - fy) * texel(tex, tw, th, ix, iy, ch)
                + fx * (1 - fy) * texel(tex, tw, th, ix + 1, iy, ch)
                + (1 - fx) * fy * texel(tex, tw, th, ix, iy + 1, ch)
                + fx * fy * texel(tex, tw, th, ix + 1, iy + 1, ch);
    }
}

/*
 * or_mesh_raster: for each listed pixel (linear index y*W+x; NULL = all),
 * brute force over every face.  tex is [th][tw][3] in [0,1] (RGB8 divided by
 * 255 by the caller).  Outputs per listed pixel: tri_id (-1 none), depth
 * (FP32 view z, +inf none), rgb[3*npix] planar (bg where none), uv[2*npix]
 * planar (0 where none), bary[3*npix] perspective-correct barycentrics, and
 * the FP32 band of the nearest-face decision:
 *   depth64   the winner's FP64 depth (+inf none);
 *   depth_tol absolute FP32 error band of that depth (face_depth_relband);
 *   tri2      the runner-up among the covering faces (-1 none);
 *   tri_margin (D64(tri2) - D64(tri)) / (tol(tri) + tol(tri2)), +inf without
 *             a runner-up: below 1 an FP32 rasteriser may pick either face.
 */
void or_mesh_raster(const double *cam, int W, int H, const double *verts, const double *uvs,
                    int nv, const int *faces, int nf, const double *tex, int tw, int th,
                    const double *bg, double znear, const int64_t *pix, int64_t npix,
                    int *tri_id, float *depth, double *rgb, double *uv, double *bary,
                    double *depth64, double *depth_tol, int *tri2, double *tri_margin) {
    (void)nv;
    face_setup *fs = (face_setup *)malloc(sizeof(face_setup) * (size_t)(nf > 0 ? nf : 1));
#pragma omp parallel for schedule(static)
    for (int f = 0; f < nf; f++) setup_face(cam, verts, faces + 3 * (int64_t)f, znear, &fs[f]);
    if (pix == NULL) npix = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < npix; q++) {
        int64_t lin = pix ? pix[q] : q;
        int x = (int)(lin % W), y = (int)(lin / W);
        int64_t px = (int64_t)x * 256 + 128, py = (int64_t)y * 256 + 128;
        /* nearest by (FP32 depth, face index), and the runner-up */
        int best = -1, second = -1;
        float bestD = INFINITY, secondD = INFINITY;
        double best64 = INFINITY, second64 = INFINITY;
        int64_t bw[3] = {0, 0, 0};
        for (int f = 0; f < nf; f++) {
            if (!fs[f].valid) continue;
            int64_t w[3];
            if (!face_covers(&fs[f], px, py, w)) continue;
            double D64 = face_depth64(&fs[f], w);
            float D = (float)D64;
            if (D < bestD) {
                second = best; secondD = bestD; second64 = best64;
                best = f; bestD = D; best64 = D64;
                bw[0] = w[0]; bw[1] = w[1]; bw[2] = w[2];
            } else if (D < secondD) {
                second = f; secondD = D; second64 = D64;
            }
        }
        tri_id[q] = best;
        depth[q] = best >= 0 ? bestD : INFINITY;
        depth64[q] = best64;
        tri2[q] = second;
        depth_tol[q] = best >= 0 ? best64 * face_depth_relband(&fs[best], px, py, best64) : 0.0;
        if (second >= 0) {
            double tol2 = second64 * face_depth_relband(&fs[second], px, py, second64);
            tri_margin[q] = (second64 - best64) / (depth_tol[q] + tol2);
        } else {
            tri_margin[q] = INFINITY;
        }
        if (best < 0) {
            for (int ch = 0; ch < 3; ch++) rgb[ch * npix + q] = bg[ch];
            uv[q] = 0; uv[npix + q] = 0;
            bary[q] = bary[npix + q] = bary[2 * npix + q] = 0;
            continue;
        }
        const int *f = faces + 3 * (int64_t)best;
        double b[3], u = 0, v = 0;
        face_bary(&fs[best], bw, b);
        for (int k = 0; k < 3; k++) {
            u += b[k] * uvs[2 * (int64_t)f[k]];
            v += b[k] * uvs[2 * (int64_t)f[k] + 1];
        }
        double c[3];
        sample_bilinear(tex, tw, th, u, v, c);
        for (int ch = 0; ch < 3; ch++) rgb[ch * npix + q] = c[ch];
        uv[q] = u; uv[npix + q] = v;
        for (int k = 0; k < 3; k++) bary[k * npix + q] = b[k];
    }
    free(fs);
}

/* Independent cross-check: FP64 Moller-Trumbore ray casting through the pixel
 * centre (no snapping); returns the nearest face along the ray (two-sided). */
void or_mesh_raycast(const double *cam, int W, int H, const double *verts, const int *faces, int nf,
                     double znear, const int64_t *pix, int64_t npix, int *tri_id, double *tz,
                     double *edge_dist_px) {
    if (pix == NULL) npix = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < npix; q++) {
        int64_t lin = pix ? pix[q] : q;
        int x = (int)(lin % W), y = (int)(lin / W);
        double d[3] = {(x + 0.5 - cam[14]) / cam[12], (y + 0.5 - cam[15]) / cam[13], 1.0};
        double best_t = INFINITY, best_e = INFINITY;
        int best = -1;
        for (int f = 0; f < nf; f++) {
            double P[3][3];
            int ok = 1;
            for (int k = 0; k < 3; k++) {
                const double *v = verts + 3 * (int64_t)faces[3 * (int64_t)f + k];
                for (int r = 0; r < 3; r++)
                    P[k][r] = cam[3 * r] * v[0] + cam[3 * r + 1] * v[1] + cam[3 * r + 2] * v[2] + cam[9 + r];
                if (!(P[k][2] > znear)) ok = 0;
            }
            if (!ok) continue;
            double e1[3], e2[3], h[3], s[3], qv[3];
            for (int r = 0; r < 3; r++) { e1[r] = P[1][r] - P[0][r]; e2[r] = P[2][r] - P[0][r]; }
            h[0] = d[1] * e2[2] - d[2] * e2[1];
            h[1] = d[2] * e2[0] - d[0] * e2[2];
            h[2] = d[0] * e2[1] - d[1] * e2[0];
            double a = e1[0] * h[0] + e1[1] * h[1] + e1[2] * h[2];
            if (fabs(a) < 1e-300) continue;
            double inv = 1.0 / a;
            for (int r = 0; r < 3; r++) s[r] = -P[0][r];
            double uu = inv * (s[0] * h[0] + s[1] * h[1] + s[2] * h[2]);
            qv[0] = s[1] * e1[2] - s[2] * e1[1];
            qv[1] = s[2] * e1[0] - s[0] * e1[2];
            qv[2] = s[0] * e1[1] - s[1] * e1[0];
            double vv = inv * (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]);
            double t = inv * (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]);
            if (uu < 0 || vv < 0 || uu + vv > 1 || !(t > 0)) continue;
            if (t < best_t) {
                best_t = t;
                best = f;
                /* distance (in barycentric units) to the nearest edge */
                double m = uu < vv ? uu : vv;
                double w = 1 - uu - vv;
                best_e = m < w ? m : w;
            }
        }
        tri_id[q] = best;
        tz[q] = best_t; /* d has unit z, so the ray parameter is the view z */
        edge_dist_px[q] = best_e;
    }
}

/* ======================================================================== */
/* Real spherical harmonics (standard orthonormal basis, Condon-Shortley     */
/* phase), index l*l + l + m for m = -l..l.                                  */
/* ======================================================================== */

static double factorial(int n) {
    double r = 1;
    for (int i = 2; i <= n; i++) r *= i;
    return r;
}

/* associated Legendre P_l^m(x), m >= 0, with the (-1)^m phase */
static double assoc_legendre(int l, int m, double x) {
    double pmm = 1.0;
    double somx2 = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x)));
    double fact = 1.0;
    for (int i = 1; i <= m; i++) { pmm *= -fact * somx2; fact += 2.0; }
    if (l == m) return pmm;
    double pmmp1 = x * (2 * m + 1) * pmm;
    if (l == m + 1) return pmmp1;
    double pll = 0;
    for (int ll = m + 2; ll <= l; ll++) {
        pll = ((2 * ll - 1) * x * pmmp1 - (ll + m - 1) * pmm) / (ll - m);
        pmm = pmmp1;
        pmmp1 = pll;
    }
    return pll;
}

/* Y[(deg+1)^2] at unit direction d */
void or_sh_basis(int deg, const double *d, double *Y) {
    double ct = d[2];
    double phi = atan2(d[1], d[0]);
    for (int l = 0; l <= deg; l++) {
        for (int m = -l; m <= l; m++) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2 * l + 1) / (4 * M_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, ct);
            double y;
            if (m > 0) y = sqrt(2.0) * K * cos(m * phi) * P;
            else if (m < 0) y = sqrt(2.0) * K * sin(am * phi) * P;
            else y = K * P;
            Y[l * l + l + m] = y;
        }
    }
}

/* ======================================================================== */
/* Gaussian projection (Eq. 1, Sec. 3.1: Sigma = R S S^T R^T,                */
/* Sigma' = J W Sigma W^T J^T)                                               */
/* ======================================================================== */

/*
 * Per Gaussian i:
 *   visible[i]   1 iff the FP32 depth key z > 0.2, det(Sigma') > 0 and every
 *                parameter (opacity if given) and the colour are finite
 *   depth[i]     FP32 depth key (defined for every Gaussian)
 *   mean2d[2i..] projected mean in pixels (continuous coordinates)
 *   cov2d[3i..]  Sigma' (xx, xy, yy) including the screen-space kernel
 *   conic[3i..]  Sigma'^{-1} (xx, xy, yy)
 *   color[3i..]  max(0, 0.5 + SH(view direction))
 *   clamped[3i+ch] 1 iff the colour channel was clamped at 0
 *   opac_scale[i] factor on the opacity (1 without the Mip-Splatting filters)
 *
 * Filters (the 3DGS defaults: filt3d NULL, kernel2d 0.3, antialias 0).
 * Mip-Splatting (Yu et al., CVPR 2024), the second Gaussian back-end the
 * paper pairs with the mesh (Tab. 1), low-passes every Gaussian twice:
 *   - 3D smoothing: Sigma + v_i I with a per-Gaussian variance v_i = filt3d[i]
 *     (from the cameras' sampling rates, see the Python front end); as R is
 *     orthonormal this is R diag(s_k^2 + v_i) R^T, and the opacity is scaled
 *     by sqrt(det Sigma / det(Sigma + v_i I)) = prod_k s_k / sqrt(s_k^2 + v_i);
 *   - 2D Mip filter: Sigma2D + kernel2d I (kernel2d 0.1, a one-pixel box
 *     approximated by a Gaussian) instead of the 0.3 dilation, and with
 *     antialias the opacity is scaled by sqrt(det Sigma2D / det(Sigma2D +
 *     kernel2d I)) (0 where det Sigma2D <= 0).
 */
void or_project(const double *cam, int W, int H, int n, const double *means, const double *scales,
                const double *quats, const double *opacity, const double *sh, int sh_degree,
                const double *filt3d,
                double kernel2d, int antialias, int *visible, float *depth, double *mean2d,
                double *cov2d, double *conic, double *color, int *clamped, double *opac_scale) {
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const double limx = 1.3 * (0.5 * W / fx), limy = 1.3 * (0.5 * H / fy);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    double C[3]; /* camera centre = -R^T t */
    for (int j = 0; j < 3; j++) C[j] = -(cam[j] * cam[9] + cam[3 + j] * cam[10] + cam[6 + j] * cam[11]);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        const double *m = means + 3 * (int64_t)i;
        double tz = view_coord(cam, 2, m[0], m[1], m[2]);
        double tx = view_coord(cam, 0, m[0], m[1], m[2]);
        double ty = view_coord(cam, 1, m[0], m[1], m[2]);
        float zf = (float)tz;
        depth[i] = zf;
        visible[i] = 0;
        mean2d[2 * i] = mean2d[2 * i + 1] = 0;
        for (int k = 0; k < 3; k++) cov2d[3 * i + k] = conic[3 * i + k] = color[3 * i + k] = 0, clamped[3 * i + k] = 0;
        opac_scale[i] = 1.0;
        if (!(zf > 0.2f)) continue;
        /* reading (the paper does not define them): a Gaussian with a
         * non-finite mean, scale, quaternion, opacity or 3D-filter variance,
         * or a zero quaternion, is culled like one behind the near plane */
        {
            const double *qq = quats + 4 * (int64_t)i, *ss = scales + 3 * (int64_t)i;
            int fin = isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]) && (!opacity || isfinite(opacity[i]));
            for (int k = 0; k < 3; k++) fin = fin && isfinite(ss[k]);
            for (int k = 0; k < 4; k++) fin = fin && isfinite(qq[k]);
            fin = fin && (qq[0] != 0 || qq[1] != 0 || qq[2] != 0 || qq[3] != 0);
            if (filt3d) fin = fin && isfinite(filt3d[i]);
            if (!fin) continue;
        }
        /* rotation from the normalised quaternion (w,x,y,z) */
        const double *q = quats + 4 * (int64_t)i;
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        double Rq[3][3] = {
            {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        const double *s = scales + 3 * (int64_t)i;
        const double v3 = filt3d ? filt3d[i] : 0.0;
        double rho3 = 1.0, s2k[3];
        for (int k = 0; k < 3; k++) {
            s2k[k] = s[k] * s[k] + v3;
            if (v3 > 0) rho3 *= s[k] / sqrt(s2k[k]);
        }
        double Sig[3][3];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0;
                for (int k = 0; k < 3; k++) acc += Rq[a][k] * s2k[k] * Rq[b][k];
                Sig[a][b] = acc;
            }
        /* J with the half-FOV clamp of the view-space x/z, y/z */
        double txz = tx / tz, tyz = ty / tz;
        if (txz < -limx) txz = -limx;
        if (txz > limx) txz = limx;
        if (tyz < -limy) tyz = -limy;
        if (tyz > limy) tyz = limy;
        double J[2][3] = {{fx / tz, 0, -fx * txz / tz}, {0, fy / tz, -fy * tyz / tz}};
        double T[2][3]; /* T = J W */
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0;
                for (int k = 0; k < 3; k++) acc += J[a][k] * cam[3 * k + b];
                T[a][b] = acc;
            }
        double S2[2][2];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                double acc = 0;
                for (int k = 0; k < 3; k++)
                    for (int l = 0; l < 3; l++) acc += T[a][k] * Sig[k][l] * T[b][l];
                S2[a][b] = acc;
            }
        double a_ = S2[0][0] + kernel2d, b_ = S2[0][1], c_ = S2[1][1] + kernel2d;
        double det = a_ * c_ - b_ * b_;
        if (!(det > 0)) continue;
        visible[i] = 1;
        double rho2 = 1.0;
        if (antialias) {
            const double det0 = S2[0][0] * S2[1][1] - S2[0][1] * S2[0][1];
            rho2 = det0 > 0 ? sqrt(det0 / det) : 0.0;
        }
        opac_scale[i] = rho3 * rho2;
        cov2d[3 * i] = a_; cov2d[3 * i + 1] = b_; cov2d[3 * i + 2] = c_;
        conic[3 * i] = c_ / det; conic[3 * i + 1] = -b_ / det; conic[3 * i + 2] = a_ / det;
        mean2d[2 * i] = fx * tx / tz + cx;
        mean2d[2 * i + 1] = fy * ty / tz + cy;
        /* colour from SH in the direction camera centre -> mean */
        double d[3] = {m[0] - C[0], m[1] - C[1], m[2] - C[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; k++) d[k] /= dn;
        double Y[16];
        or_sh_basis(sh_degree, d, Y);
        for (int ch = 0; ch < 3; ch++) {
            double acc = 0.5;
            for (int k = 0; k < K; k++) acc += Y[k] * sh[((int64_t)i * K + k) * 3 + ch];
            clamped[3 * i + ch] = acc < 0;
            color[3 * i + ch] = acc < 0 ? 0 : acc;
            if (!isfinite(acc)) visible[i] = 0;       /* non-finite SH: culled (same reading) */
        }
    }
}

/* ======================================================================== */
/* Hybrid blending (Eq. 2 and the joint-rasterisation composite of Sec. 3.4) */
/* ======================================================================== */

static const double *g_sort_depth_base;
static int cmp_depth_index(const void *pa, const void *pb) {
    int a = *(const int *)pa, b = *(const int *)pb;
    float da = ((const float *)g_sort_depth_base)[a], db = ((const float *)g_sort_depth_base)[b];
    if (da < db) return -1;
    if (da > db) return 1;
    return (a > b) - (a < b);
}

/* visible Gaussians sorted by (FP32 depth, index) ascending */
int or_sort_order(int n, const int *visible, const float *depth, int *order) {
    int m = 0;
    for (int i = 0; i < n; i++)
        if (visible[i]) order[m++] = i;
    g_sort_depth_base = (const double *)depth;
    qsort(order, (size_t)m, sizeof(int), cmp_depth_index);
    return m;
}

typedef struct {
    double rgb[3], T, margin;
    int n_contrib, n_amb;
    int64_t evaluated;
    uint64_t fp;
} px_result;

static uint64_t mix64(uint64_t h, uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h * 0xBF58476D1CE4E5B9ull;
}

/*
 * Ambiguity band (tolerance model, not part of the rendered result).  The
 * decisions of the walk are exact here (FP64); a renderer that takes them in
 * FP32 (u = 2^-24) sees each value moved by at most:
 *   projected mean  |dm_x| <= 2u (|m_x - c_x| + |m_x|): twice the half-ulp
 *                   roundings of the ratio x/z and of the FMA with f_x and
 *                   c_x, the same for y;
 *   conic           every element within (16 kappa_c) u relative, kappa_c =
 *                   sqrt(lambda_max / lambda_min) of Sigma' (Sigma' is formed
 *                   from its square root V V^T, so the error of the small
 *                   eigenvalue scales with sqrt(lambda_max lambda_min));
 *   d^2             |dd2| <= 2 (|g_x| dm_x + |g_y| dm_y) + (16 kappa_c + 4) u S,
 *                   g = conic (p - m), S = sum of |terms| of d^2;
 *   alpha           |da| <= alpha (|dd2| / 2 + 16 u) (exp, opacity factors);
 *                   the 0.99 clamp held in FP32 is 0.99 + 9.5e-9;
 *   T' = T (1 - a)  relative error sum over the blended j of
 *                   2u + |da_j| / (1 - a_j);
 *   mesh cut        D_m within the mesh pass's depth band (or_mesh_raster);
 *                   the cut of a Gaussian in that band can change the pixel
 *                   only if it, or a later Gaussian still in the band, could
 *                   be blended there (d^2 and alpha within their bands of
 *                   passing), so only then is it counted.
 * A decision whose value lies within `band` times that bound of its threshold
 * is ambiguous: it counts in n_amb and its margin (distance / bound) is below
 * 1.  The d^2 test counts only where it can matter (o e^-4.5 >= 1/255: below
 * that a Gaussian on the ellipse fails the alpha test either way).
 *
 * or_blend_errscale: per Gaussian the three scales of that model,
 * err[3i..] = (dm_x, dm_y, kappa_c); zeros for invisible Gaussians.
 */
#define OR_U 0x1p-24

void or_blend_errscale(const double *cam, int n, const int *visible, const double *mean2d,
                       const double *cov2d, double *err) {
    const double cx = cam[14], cy = cam[15];
    for (int i = 0; i < n; i++) {
        err[3 * i] = err[3 * i + 1] = err[3 * i + 2] = 0.0;
        if (!visible[i]) continue;
        double mx = mean2d[2 * i], my = mean2d[2 * i + 1];
        err[3 * i] = 2.0 * OR_U * (fabs(mx - cx) + fabs(mx));
        err[3 * i + 1] = 2.0 * OR_U * (fabs(my - cy) + fabs(my));
        double a = cov2d[3 * i], b = cov2d[3 * i + 1], c = cov2d[3 * i + 2];
        double h = 0.5 * (a + c), r = sqrt(0.25 * (a - c) * (a - c) + b * b);
        double lmin = h - r, lmax = h + r;
        err[3 * i + 2] = lmin > 0 ? sqrt(lmax / lmin) : INFINITY;
    }
}

/* one decision of the walk: returns its outcome, inverted when it is the
 * j-th ambiguous decision met on this walk and bit j of `flip` is set */
static int decide(int outcome, double margin, uint32_t flip, int *namb, double *mmin) {
    if (margin < *mmin) *mmin = margin;
    if (margin < 1.0) {
        int j = (*namb)++;
        if (j < 32 && ((flip >> j) & 1u)) outcome = !outcome;
    }
    return outcome;
}

/* Band of d^2 at the pixel for Gaussian i (see the model above); *d2 gets d^2. */
static double d2_band(double pxc, double pyc, int i, const double *mean2d, const double *conic,
                      const double *err, double *d2) {
    const double *co = conic + 3 * i;
    double dx = pxc - mean2d[2 * i], dy = pyc - mean2d[2 * i + 1];
    *d2 = co[0] * dx * dx + 2.0 * co[1] * dx * dy + co[2] * dy * dy;
    double gx = co[0] * dx + co[1] * dy, gy = co[1] * dx + co[2] * dy;
    double Sabs = fabs(co[0]) * dx * dx + 2.0 * fabs(co[1] * dx * dy) + fabs(co[2]) * dy * dy;
    return 2.0 * (fabs(gx) * err[3 * i] + fabs(gy) * err[3 * i + 1])
         + (16.0 * err[3 * i + 2] + 4.0) * OR_U * Sabs;
}

/* could an FP32 evaluation blend Gaussian i at the pixel? */
static int maybe_blended(double pxc, double pyc, int i, const double *mean2d, const double *conic,
                         const double *opacity, const double *err, double band) {
    double d2, bd2 = band * d2_band(pxc, pyc, i, mean2d, conic, err, &d2);
    double dmin = d2 - bd2 > 0.0 ? d2 - bd2 : 0.0;
    if (dmin > 9.0) return 0;
    double amax = opacity[i] * exp(-0.5 * dmin) * (1.0 + band * 16.0 * OR_U);
    return amax >= 1.0 / 255.0;
}

/* Blend one pixel over the (depth, index)-sorted list `lst` (length m):
 * Eq. 2 front to back with the Sec. 3.4 cut at the mesh depth.  Dm is the
 * FP32 mesh depth the cut compares with; Dm64 and Dtol its FP64 value and
 * band.  flip: see decide(). */
static void blend_pixel(double pxc, double pyc, int hit, float Dm, double Dm64, double Dtol,
                        const double *Im, const int *lst, int m, const float *depth,
                        const double *mean2d, const double *conic, const double *opacity,
                        const double *color, const double *err, double band, uint32_t flip,
                        px_result *r) {
    double T = 1.0, C[3] = {0, 0, 0}, margin = INFINITY, relT = 0.0;
    int n = 0, namb = 0;
    int64_t ev = 0;
    uint64_t fp = 1469598103934665603ull;
    const double a_min = 1.0 / 255.0;
    for (int j = 0; j < m; j++) {
        int i = lst[j];
        if (hit) {                                    /* behind the mesh: stop (not hashed) */
            double mc = fabs((double)depth[i] - Dm64) / (band * Dtol);
            if (mc < 1.0) {
                /* in the band: it matters only if this or a later Gaussian
                 * of the band could be blended here */
                int matters = 0;
                for (int k = j; k < m && !matters; k++) {
                    if ((double)depth[lst[k]] > Dm64 + band * Dtol) break;
                    matters = maybe_blended(pxc, pyc, lst[k], mean2d, conic, opacity, err, band);
                }
                if (!matters) mc = INFINITY;
            }
            if (decide(depth[i] >= Dm, mc, flip, &namb, &margin)) break;
        }
        double d2, bd2 = d2_band(pxc, pyc, i, mean2d, conic, err, &d2);
        double md = opacity[i] * exp(-4.5) * (1.0 + 1e-4) >= a_min ? fabs(d2 - 9.0) / (band * bd2)
                                                                 : INFINITY;
        if (decide(d2 > 9.0, md, flip, &namb, &margin)) continue;   /* outside the 3-sigma ellipse */
        ev++;
        double araw = opacity[i] * exp(-0.5 * d2);
        double ba = araw * (0.5 * bd2 + 16.0 * OR_U);
        if (decide(araw < a_min, fabs(araw - a_min) / (band * ba), flip, &namb, &margin))
            continue;                                 /* too transparent */
        int clamp99 = araw > 0.99;
        double a = clamp99 ? 0.99 : araw;
        relT += 2.0 * OR_U + (clamp99 ? 1e-8 : ba) / (1.0 - a);
        double Tn = T * (1.0 - a);
        if (decide(Tn < 1e-4, fabs(Tn - 1e-4) / (band * Tn * relT), flip, &namb, &margin)) {
            fp = mix64(fp, 0x57097ull);               /* saturated */
            break;
        }
        for (int ch = 0; ch < 3; ch++) C[ch] += a * T * color[3 * i + ch];
        T = Tn;
        n++;
        fp = mix64(fp, (uint64_t)i * 2 + (uint64_t)clamp99);
    }
    for (int ch = 0; ch < 3; ch++) r->rgb[ch] = C[ch] + T * Im[ch];
    r->T = T;
    r->n_contrib = n;
    r->n_amb = namb;
    r->margin = margin;
    r->evaluated = ev;
    r->fp = fp;
}

/*
 * or_blend: per listed pixel (NULL = all W*H), walk `order` (all visible
 * Gaussians sorted by depth then index: brute force).  mesh_rgb is planar
 * [3][npix] per listed pixel; tri_id, mesh_depth (FP32), mesh_depth64 and
 * mesh_tol per listed pixel (tri_id < 0: no triangle, use bg).  err: the
 * per-Gaussian scales of or_blend_errscale; band scales the ambiguity band.
 * Outputs: rgb planar [3][npix], T, n_contrib, n_amb (ambiguous decisions),
 * margin (smallest decision margin in units of its band), evaluated (alpha
 * evaluations), fp (hash of the pixel's decisions).
 */
void or_blend(int W, int H, int n, const int *order, int m, const float *depth,
              const double *mean2d, const double *conic, const double *opacity,
              const double *color, const double *err, const int *tri_id, const float *mesh_depth,
              const double *mesh_depth64, const double *mesh_tol, const double *mesh_rgb,
              const double *bg, double band, const int64_t *pix, int64_t npix, double *rgb,
              double *T, int *n_contrib, int *n_amb, double *margin, int64_t *evaluated,
              uint64_t *fp) {
    (void)n; (void)H;
    if (pix == NULL) npix = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; q++) {
        int64_t lin = pix ? pix[q] : q;
        int x = (int)(lin % W), y = (int)(lin / W);
        int hit = tri_id[q] >= 0;
        double Im[3];
        for (int ch = 0; ch < 3; ch++) Im[ch] = hit ? mesh_rgb[ch * npix + q] : bg[ch];
        px_result r;
        blend_pixel(x + 0.5, y + 0.5, hit, mesh_depth[q], mesh_depth64[q], mesh_tol[q], Im, order,
                    m, depth, mean2d, conic, opacity, color, err, band, 0u, &r);
        for (int ch = 0; ch < 3; ch++) rgb[ch * npix + q] = r.rgb[ch];
        T[q] = r.T;
        n_contrib[q] = r.n_contrib;
        n_amb[q] = r.n_amb;
        margin[q] = r.margin;
        evaluated[q] = r.evaluated;
        fp[q] = r.fp;
    }
}

/*
 * or_blend_flipped: one pixel (x, y) walked with the ambiguous decisions
 * selected by `flip` inverted (bit j: the j-th ambiguous decision met on the
 * walk).  Over the flip masks this lists every outcome an FP32 renderer may
 * validly produce at an ambiguous pixel.  Im: the pixel's mesh colour (or
 * bg); out: rgb[3], T, n_contrib, n_amb.
 */
void or_blend_flipped(int x, int y, const int *order, int m, const float *depth,
                      const double *mean2d, const double *conic, const double *opacity,
                      const double *color, const double *err, int hit, float Dm, double Dm64,
                      double Dtol, const double *Im, double band, uint32_t flip, double *rgb,
                      double *T, int *n_contrib, int *n_amb) {
    px_result r;
    blend_pixel(x + 0.5, y + 0.5, hit, Dm, Dm64, Dtol, Im, order, m, depth, mean2d, conic,
                opacity, color, err, band, flip, &r);
    for (int ch = 0; ch < 3; ch++) rgb[ch] = r.rgb[ch];
    *T = r.T;
    *n_contrib = r.n_contrib;
    *n_amb = r.n_amb;
}

/*
 * or_blend_grid: the same per-pixel walk for full images, with an exact
 * prefilter.  Each visible Gaussian is listed in every cell (cell x cell px)
 * touched by the rectangle of its ellipse d^2 <= 9 (1 + 1e-2), inflated by
 * 1 px; a pixel then walks only its cell's list, which keeps the global
 * (depth, index) order.  Every Gaussian that could pass or come near the
 * d^2 <= 9 test at a pixel is in that pixel's list, so results, decision
 * hashes and every d^2 margin whose band is below 1e-2 relative (the band
 * of or_blend_errscale stays far below that: sigma' >= 0.55 px after the
 * dilation) are identical to or_blend.  Inputs/outputs as or_blend with
 * full images (pixel q = y*W+x), mesh_rgb planar [3][W*H].
 */
void or_blend_grid(int W, int H, int cell, const int *order, int m, const float *depth,
                   const double *mean2d, const double *cov2d, const double *conic,
                   const double *opacity, const double *color, const double *err,
                   const int *tri_id, const float *mesh_depth, const double *mesh_depth64,
                   const double *mesh_tol, const double *mesh_rgb, const double *bg, double band,
                   int row0, int row1, double *rgb, double *T, int *n_contrib, int *n_amb,
                   double *margin, int64_t *evaluated, uint64_t *fp) {
    int gw = (W + cell - 1) / cell, gh = (H + cell - 1) / cell;
    int64_t ncell = (int64_t)gw * gh;
    int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int *rx0 = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1) * 4);
    const double k = 3.0 * sqrt(1.0 + 1e-2);
    for (int j = 0; j < m; j++) {
        int i = order[j];
        double hx = k * sqrt(cov2d[3 * i]) + 1.0, hy = k * sqrt(cov2d[3 * i + 2]) + 1.0;
        double x0 = floor((mean2d[2 * i] - hx) / cell), x1 = floor((mean2d[2 * i] + hx) / cell);
        double y0 = floor((mean2d[2 * i + 1] - hy) / cell), y1 = floor((mean2d[2 * i + 1] + hy) / cell);
        /* clamp in FP64 before converting: far off-screen means are huge */
        int ax0 = (int)fmin(fmax(0.0, x0), (double)gw), ax1 = (int)fmax(fmin(gw - 1.0, x1), -1.0);
        int ay0 = (int)fmin(fmax(0.0, y0), (double)gh), ay1 = (int)fmax(fmin(gh - 1.0, y1), -1.0);
        rx0[4 * j] = ax0; rx0[4 * j + 1] = ax1; rx0[4 * j + 2] = ay0; rx0[4 * j + 3] = ay1;
        for (int cy = ay0; cy <= ay1; cy++)
            for (int cx = ax0; cx <= ax1; cx++) cnt[(int64_t)cy * gw + cx + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) cnt[c + 1] += cnt[c];
    int *lists = (int *)malloc(sizeof(int) * (size_t)(cnt[ncell] > 0 ? cnt[ncell] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)ncell);
    for (int j = 0; j < m; j++) {
        for (int cy = rx0[4 * j + 2]; cy <= rx0[4 * j + 3]; cy++)
            for (int cx = rx0[4 * j]; cx <= rx0[4 * j + 1]; cx++) lists[fill[(int64_t)cy * gw + cx]++] = order[j];
    }
    int64_t npx = (int64_t)W * H;
    if (row1 > H) row1 = H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = row0; y < row1; y++) {
        for (int x = 0; x < W; x++) {
            int64_t q = (int64_t)y * W + x;
            int64_t c = (int64_t)(y / cell) * gw + (x / cell);
            int hit = tri_id[q] >= 0;
            double Im[3];
            for (int ch = 0; ch < 3; ch++) Im[ch] = hit ? mesh_rgb[ch * npx + q] : bg[ch];
            px_result r;
            blend_pixel(x + 0.5, y + 0.5, hit, mesh_depth[q], mesh_depth64[q], mesh_tol[q], Im,
                        lists + cnt[c], (int)(cnt[c + 1] - cnt[c]), depth, mean2d, conic, opacity,
                        color, err, band, 0u, &r);
            for (int ch = 0; ch < 3; ch++) rgb[ch * npx + q] = r.rgb[ch];
            T[q] = r.T;
            n_contrib[q] = r.n_contrib;
            n_amb[q] = r.n_amb;
            margin[q] = r.margin;
            evaluated[q] = r.evaluated;
            fp[q] = r.fp;
        }
    }
    free(cnt); free(rx0); free(lists); free(fill);
}
