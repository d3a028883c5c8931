// mesh_raster.cu -- textured-mesh rasterisation (Sec. 3.1 "Textured mesh":
// barycentric UV interpolation and a texture lookup per pixel) producing the
// I_m and D_m of the joint rasterisation (Sec. 3.4).
//
// Pipeline (all cameras of a call at once):
//   vertex pass   FP64 view transform (fixed FMA order), projection, snap to
//                 1/256 px, 1/z;
//   face pass     orientation, bounding box, the tiles it touches (atomic
//                 per-tile face counts);
//   scan + emit   per-tile offsets; each face's index into the bucket of
//                 every tile it touches (atomic slots: the order within a
//                 bucket does not matter);
//   tile pass     one CTA per tile, a thread per two adjacent pixels of a row:
//                 for every face of the tile's bucket, exact int64 edge
//                 functions with the top-left rule at the pixel centres; the
//                 face's affine 1/z in FP32, packed with the inverted face
//                 index into a signed 64-bit key whose maximum over the faces
//                 is (largest FP32 1/z, lowest face index) whatever the
//                 bucket order; the depth is the FP32 reciprocal of the
//                 winner's 1/z (one division per pixel, not per face); then
//                 the resolve: perspective-
//                 correct UVs, bilinear clamp-to-edge texel fetch, outputs
//                 and the tile's farthest mesh depth (for the Gaussian pair
//                 cull).  No per-pixel visibility buffer and no global
//                 atomics on pixels.
#include <limits.h>

#include "hm_host.h"

namespace hm {

namespace {

constexpr double kSnap = 256.0;
constexpr double kGuard = 2097152.0;   // 2^21 px
constexpr int kInvalid = INT_MIN;

// 16-byte aligned, with the fields a pass reads together in whole 16-byte
// chunks (coverage: x, y, flip, plane; resolve: x, y, izf, rD, uv)
struct __align__(16) FaceSetup {
    int x[3], y[3];          // snapped positions in the face's vertex order
    int flip;                // signed area negative: traverse 0 -> 2 -> 1
    float iz0f, af, bf;      // 1/z = iz0 + a U + b V, (U,V) = centre - vertex 0 in pixels
    float izf[3];            // 1 / view z per vertex (FP32)
    float rD;                // 1 / signed double area
    float u0, v0, du1, dv1, du2, dv2;   // uv0 and uv_k - uv0
    int tx0, tx1, ty0, ty1;  // touched tiles (empty: tx0 > tx1)
    long long area2;         // |signed double area| (1/256 px)^2
};
static_assert(sizeof(FaceSetup) == 112, "face set-up layout");

__global__ void __launch_bounds__(256)
mesh_vertex_kernel(ViewTable vt, int nv, const float *__restrict__ verts, double znear,
                   int2 *__restrict__ sxy, double *__restrict__ iz) {
    const long long m = (long long)vt.n_views * nv;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < m;
         it += (long long)gridDim.x * blockDim.x) {
        const int v = (int)((uint32_t)it / (uint32_t)nv);   // m < 2^31
        const long long k = it - (long long)v * nv;
        const ViewDev &V = vt.v[v];
        const double x = verts[3 * k], y = verts[3 * k + 1], z = verts[3 * k + 2];
        const double X = fma((double)V.R[0], x, fma((double)V.R[1], y, fma((double)V.R[2], z, (double)V.t[0])));
        const double Y = fma((double)V.R[3], x, fma((double)V.R[4], y, fma((double)V.R[5], z, (double)V.t[1])));
        const double Z = fma((double)V.R[6], x, fma((double)V.R[7], y, fma((double)V.R[8], z, (double)V.t[2])));
        int2 o = make_int2(kInvalid, kInvalid);
        double r = 0.0;
        if (Z > znear) {
            const double sx = fma((double)V.fx, X / Z, (double)V.cx);
            const double sy = fma((double)V.fy, Y / Z, (double)V.cy);
            if (fabs(sx) <= kGuard && fabs(sy) <= kGuard) {
                o.x = (int)__double2ll_rn(sx * kSnap);
                o.y = (int)__double2ll_rn(sy * kSnap);
                r = 1.0 / Z;
            }
        }
        sxy[it] = o;
        iz[it] = r;
    }
}

__device__ __forceinline__ long long floor_div(long long a, long long b) {
    long long q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__global__ void __launch_bounds__(256)
mesh_face_kernel(ViewTable vt, int nv, int nf, const int32_t *__restrict__ faces,
                 const float *__restrict__ uvs, const int2 *__restrict__ sxy,
                 const double *__restrict__ iz, FaceSetup *__restrict__ setup,
                 uint32_t *__restrict__ tile_fcnt) {
    const long long m = (long long)vt.n_views * nf;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < m;
         it += (long long)gridDim.x * blockDim.x) {
        const int v = (int)((uint32_t)it / (uint32_t)nf);   // m < 2^31
        const long long f = it - (long long)v * nf;
        const ViewDev &V = vt.v[v];
        FaceSetup s;
        s.tx0 = 1; s.tx1 = 0; s.ty0 = 1; s.ty1 = 0;
        s.flip = 0; s.area2 = 0;
        s.iz0f = s.af = s.bf = s.rD = 0.f;
        double izd[3];
        float fu[3] = {0.f, 0.f, 0.f}, fv[3] = {0.f, 0.f, 0.f};
        bool ok = true;
        for (int k = 0; k < 3; ++k) {
            const int vi = faces[3 * f + k];
            s.izf[k] = 0.f;
            izd[k] = 0.0;
            if (vi < 0 || vi >= nv) { ok = false; s.x[k] = s.y[k] = 0; continue; }
            fu[k] = uvs[2 * (long long)vi];
            fv[k] = uvs[2 * (long long)vi + 1];
            const int2 p = sxy[(long long)v * nv + vi];
            s.x[k] = p.x; s.y[k] = p.y;
            izd[k] = iz[(long long)v * nv + vi];
            s.izf[k] = __double2float_rn(izd[k]);
            if (p.x == kInvalid) ok = false;
        }
        s.u0 = fu[0]; s.v0 = fv[0];
        s.du1 = fu[1] - fu[0]; s.dv1 = fv[1] - fv[0];
        s.du2 = fu[2] - fu[0]; s.dv2 = fv[2] - fv[0];
        if (ok) {
            const long long e1x = (long long)s.x[1] - s.x[0], e1y = (long long)s.y[1] - s.y[0];
            const long long e2x = (long long)s.x[2] - s.x[0], e2y = (long long)s.y[2] - s.y[0];
            const long long a2 = e1x * e2y - e1y * e2x;
            if (a2 != 0) {
                s.flip = a2 < 0;
                s.area2 = a2 < 0 ? -a2 : a2;
                // screen-space barycentrics of the offset (dx,dy) from vertex 0 (Cramer):
                // l1 = (dx e2y - dy e2x)/D, l2 = (e1x dy - e1y dx)/D, so
                // 1/z = iz0 + (iz1-iz0) l1 + (iz2-iz0) l2 = iz0 + a dx + b dy
                const double d1 = izd[1] - izd[0], d2 = izd[2] - izd[0];
                const double na = fma(d1, (double)e2y, -(d2 * (double)e1y));
                const double nb = fma(d2, (double)e1x, -(d1 * (double)e2x));
                // one FP64 division: 256 / a2 (a power-of-two multiple of 1 / a2)
                const double inv = 256.0 / (double)a2;
                s.af = __double2float_rn(na * inv);
                s.bf = __double2float_rn(nb * inv);
                s.iz0f = __double2float_rn(izd[0]);
                s.rD = __double2float_rn(inv * (1.0 / 256.0));
                const long long mnx = min(s.x[0], min(s.x[1], s.x[2])), mxx = max(s.x[0], max(s.x[1], s.x[2]));
                const long long mny = min(s.y[0], min(s.y[1], s.y[2])), mxy = max(s.y[0], max(s.y[1], s.y[2]));
                // pixel centres 256 x + 128 inside [mn, mx]
                long long x0 = -floor_div(-(mnx - 128), 256), x1 = floor_div(mxx - 128, 256);
                long long y0 = -floor_div(-(mny - 128), 256), y1 = floor_div(mxy - 128, 256);
                x0 = max(x0, 0ll); x1 = min(x1, (long long)V.W - 1);
                y0 = max(y0, 0ll); y1 = min(y1, (long long)V.H - 1);
                if (x0 <= x1 && y0 <= y1) {
                    // (clamped to the image: 32-bit divisions)
                    s.tx0 = (int)x0 / vt.tile_w; s.tx1 = (int)x1 / vt.tile_w;
                    s.ty0 = (int)y0 / vt.tile_h; s.ty1 = (int)y1 / vt.tile_h;
                    for (int ty = s.ty0; ty <= s.ty1; ++ty)
                        for (int tx = s.tx0; tx <= s.tx1; ++tx)
                            atomicAdd(&tile_fcnt[V.tile_off + ty * V.tiles_x + tx], 1u);
                }
            }
        }
        setup[it] = s;
    }
}

// each face's index into the bucket of every tile it touches; nothing when
// the item capacity was exceeded (*n_items == 0)
__global__ void __launch_bounds__(256)
mesh_emit_kernel(ViewTable vt, int nf, const FaceSetup *__restrict__ setup, const long long *n_items,
                 uint32_t *__restrict__ cursor, uint32_t *__restrict__ items) {
    if (*n_items == 0) return;
    const long long m = (long long)vt.n_views * nf;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < m;
         it += (long long)gridDim.x * blockDim.x) {
        const FaceSetup &s = setup[it];
        if (s.tx0 > s.tx1) continue;
        const ViewDev &V = vt.v[(int)((uint32_t)it / (uint32_t)nf)];
        const int nx = s.tx1 - s.tx0 + 1, nt = nx * (s.ty1 - s.ty0 + 1);
        const uint32_t g0 = V.tile_off + s.ty0 * V.tiles_x + s.tx0;
        // slots four at a time (independent atomics in flight together), then the stores
        for (int b0 = 0; b0 < nt; b0 += 4) {
            uint32_t pos[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (b0 + q < nt) {
                    const uint32_t tile = g0 + ((b0 + q) / nx) * V.tiles_x + (b0 + q) % nx;
                    pos[q] = hm_check(tile < (uint32_t)vt.total_tiles) ? atomicAdd(&cursor[tile], 1u) : ~0u;
                }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (b0 + q < nt && hm_check(pos[q] < (unsigned long long)*n_items)) items[pos[q]] = (uint32_t)it;
        }
    }
}

// texture coordinates and bilinear weights of a covered pixel centre
struct TexTap {
    float u, w;          // perspective-correct UV
    int x0, x1, y0, y1;  // clamped texel columns and rows
    float w00, w10, w01, w11;
};

// what the resolve of a covered pixel needs of its face
struct TexFace {
    int x0, y0;                 // snapped vertex 0
    float e1x, e1y, e2x, e2y;   // snapped edges from vertex 0 (exact integers, rounded to FP32 once)
    float rD, izf1, izf2;       // 1 / signed double area, 1/z of vertices 1 and 2
    float u0, v0, du1, dv1, du2, dv2;
};

// (snapped coordinates stay within +-2^29, so the differences fit int32)
__device__ __forceinline__ TexFace tex_face(const FaceSetup &g) {
    TexFace f;
    f.x0 = g.x[0]; f.y0 = g.y[0];
    f.e1x = __int2float_rn(g.x[1] - g.x[0]); f.e1y = __int2float_rn(g.y[1] - g.y[0]);
    f.e2x = __int2float_rn(g.x[2] - g.x[0]); f.e2y = __int2float_rn(g.y[2] - g.y[0]);
    f.rD = g.rD; f.izf1 = g.izf[1]; f.izf2 = g.izf[2];
    f.u0 = g.u0; f.v0 = g.v0; f.du1 = g.du1; f.dv1 = g.dv1; f.du2 = g.du2; f.dv2 = g.dv2;
    return f;
}

__device__ __forceinline__ TexTap tex_tap(const TexFace &s, int px, int py, float D, int tw, int th) {
    TexTap r;
    // perspective-correct barycentrics b_k = l_k (1/z_k) z, l_k the
    // screen-space ones of the offset from vertex 0 (Cramer's rule)
    const float dx = __int2float_rn(px * 256 + 128 - s.x0);
    const float dy = __int2float_rn(py * 256 + 128 - s.y0);
    const float e1x = s.e1x, e1y = s.e1y, e2x = s.e2x, e2y = s.e2y;
    const float l1 = fmaf(dx, e2y, -dy * e2x) * s.rD;
    const float l2 = fmaf(e1x, dy, -e1y * dx) * s.rD;
    const float b1 = l1 * s.izf1 * D, b2 = l2 * s.izf2 * D;
    // uv = uv0 + b1 (uv1 - uv0) + b2 (uv2 - uv0): the corrections are small
    // for small faces, so uv keeps close to FP32 rounding of its value
    r.u = s.u0 + fmaf(b1, s.du1, b2 * s.du2);
    r.w = s.v0 + fmaf(b1, s.dv1, b2 * s.dv2);
    const float ss = r.u * (float)tw - 0.5f, tt = r.w * (float)th - 0.5f;
    const float xf = floorf(ss), yf = floorf(tt);
    const float fx = ss - xf, fy = tt - yf;
    const int ix = (int)fmaxf(fminf(xf, 1e8f), -1e8f), iy = (int)fmaxf(fminf(yf, 1e8f), -1e8f);
    // clamp-to-edge addressing
    r.x0 = min(max(ix, 0), tw - 1);
    r.x1 = min(max(ix + 1, 0), tw - 1);
    r.y0 = min(max(iy, 0), th - 1);
    r.y1 = min(max(iy + 1, 0), th - 1);
    r.w00 = (1.f - fx) * (1.f - fy);
    r.w10 = fx * (1.f - fy);
    r.w01 = (1.f - fx) * fy;
    r.w11 = fx * fy;
    return r;
}

// bilinear clamp-to-edge fetch: the four texels' channels are read at
// immediate offsets from per-texel base pointers (RGB8: the byte values);
// the mix sums the weighted values and, for RGB8, scales by 1/255 once per
// channel
template <bool F32TEX>
__device__ __forceinline__ void texels(const void *tex, int tw, const TexTap &a, float (&tv)[4][3]) {
    const size_t r0 = (size_t)a.y0 * (size_t)tw * 3, r1 = (size_t)a.y1 * (size_t)tw * 3;
    const int x0 = a.x0 * 3, x1 = a.x1 * 3;
    if (F32TEX) {
        const float *T = reinterpret_cast<const float *>(tex);
        const float *p00 = T + r0 + x0, *p10 = T + r0 + x1, *p01 = T + r1 + x0, *p11 = T + r1 + x1;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            tv[0][ch] = __ldg(p00 + ch);
            tv[1][ch] = __ldg(p10 + ch);
            tv[2][ch] = __ldg(p01 + ch);
            tv[3][ch] = __ldg(p11 + ch);
        }
    } else {
        const unsigned char *T = reinterpret_cast<const unsigned char *>(tex);
        const unsigned char *p00 = T + r0 + x0, *p10 = T + r0 + x1, *p01 = T + r1 + x0, *p11 = T + r1 + x1;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            tv[0][ch] = (float)__ldg(p00 + ch);
            tv[1][ch] = (float)__ldg(p10 + ch);
            tv[2][ch] = (float)__ldg(p01 + ch);
            tv[3][ch] = (float)__ldg(p11 + ch);
        }
    }
}

template <bool F32TEX>
__device__ __forceinline__ void bilinear_mix(const TexTap &a, const float (&tv)[4][3], float *c) {
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float s = a.w00 * tv[0][ch] + a.w10 * tv[1][ch] + a.w01 * tv[2][ch] + a.w11 * tv[3][ch];
        c[ch] = F32TEX ? s : s * (1.0f / 255.0f);
    }
}

// What the coverage test of a tile needs of a face, prepared once per
// (tile, face).  Edge k of the positively oriented face has the exact
// integer function E_k(P) = dx_k (PY - ay_k) - dy_k (PX - ax_k) (1/256 px
// units), biased by -1 on edges that are not top or left, so that a pixel
// centre is covered by the edge iff E_k >= 0.  With P = O + (DX, DY), O the
// tile's first pixel centre, E_k(P) = E_k(O) + (dx_k DY - dy_k DX).  When
// every |dx|, |dy| < 2^17 (edges under 512 px), the offset term is below
// 2^30 in magnitude for any pixel of the tile, so E_k(P) >= 0 reduces to the
// int32 test (dx_k DY - dy_k DX) >= thr_k with thr_k = -E_k(O) clamped to
// int32 (if |E_k(O)| >= 2^31 its sign decides alone, and the clamp keeps
// that).  Larger faces take the exact int64 evaluation.
// (16-byte aligned; what the int32 test reads fills the first 64 bytes)
struct __align__(16) CoverFace {
    int dx[3], dy[3];   // edge vectors
    int thr[3];         // small faces: int32 thresholds
    int x0, y0;         // snapped vertex 0 (depth plane origin)
    uint32_t f;
    float af, bf, iz0f;
    int small;          // the int32 test applies
    long long e0[3];    // E_k(O), exact
};

// One CTA per screen tile; a thread owns two horizontally adjacent pixels of
// one row (x, x + 1): it finds their nearest faces among the tile's bucket
// (the plane's b V + 1/z0 term is shared by the pair), then resolves both --
// one texel fetch when both sample the same four texels, as they mostly do
// where the texture is magnified -- and stores the pair's G-buffer entries
// as 8-byte vectors when they are aligned.
template <int TW, int TH, bool F32TEX>
__global__ void __launch_bounds__(TW *TH / 2, 10)
mesh_tile_kernel(ViewTable vt, int nf, const FaceSetup *__restrict__ setup,
                 const uint32_t *__restrict__ tile_foff, const uint32_t *__restrict__ tile_fcnt,
                 const long long *n_items, const uint32_t *__restrict__ items,
                 const void *__restrict__ tex, int tw, int th, float bg0, float bg1, float bg2,
                 int32_t *__restrict__ tri_id, float *__restrict__ depth, float *__restrict__ rgb,
                 float *__restrict__ uv_out, float *__restrict__ tile_max) {
    static_assert(TW % 2 == 0, "pixel pairs along a row");
    constexpr int NT = TW * TH / 2;
    __shared__ float s_max[NT / 32];
    __shared__ CoverFace s_face[NT];
    __shared__ TexFace s_tex[NT];
    const int gt = blockIdx.x;
    const int v = view_of_tile(vt, gt);
    const ViewDev &V = vt.v[v];
    const int local = gt - V.tile_off;
    const int tx = local % V.tiles_x, ty = local / V.tiles_x;
    const int t = threadIdx.x;
    const int lx = (t % (TW / 2)) * 2, ly = t / (TW / 2);   // pixel a's place in the tile
    const int px = tx * TW + lx, py = ty * TH + ly;         // pixel a; pixel b is (px + 1, py)
    const long long npx = (long long)V.W * V.H;
    const bool in[2] = {px < V.W && py < V.H, px + 1 < V.W && py < V.H};
    const long long lp = (long long)py * V.W + px;
    long long key[2] = {LLONG_MIN, LLONG_MIN};     // no face
    uint32_t slot[2] = {0u, 0u};                   // bucket position of the key's face
    // coverage: every face of the bucket against both pixel centres.  The
    // faces' edge and depth data are staged in shared memory NT at a time
    // (one face per thread, loads in parallel), then every thread walks them.
    const uint32_t fc = *n_items > 0 ? tile_fcnt[gt] : 0u, f0 = tile_foff[gt];
    const int PX = px * 256 + 128, PY = py * 256 + 128;
    const int DX = lx * 256, DY = ly * 256;         // offset from the tile's first pixel centre
    for (uint32_t r0 = 0; r0 < fc; r0 += NT) {
        const int nb = (int)min((uint32_t)NT, fc - r0);
        __syncthreads();                             // the previous round's faces are consumed
        if (t < nb) {
            uint32_t vf = items[f0 + r0 + t];
            // (checked build: an item beyond the faces stages face 0)
            if (!hm_check(f0 + r0 + t < (unsigned long long)*n_items && vf < (uint32_t)vt.n_views * (uint32_t)nf))
                vf = 0;
            const FaceSetup g = setup[vf];
            const int b = g.flip ? 2 : 1, c = g.flip ? 1 : 2;   // oriented order 0, b, c
            const int ax[3] = {g.x[0], g.x[b], g.x[c]}, ay[3] = {g.y[0], g.y[b], g.y[c]};
            const int bx[3] = {g.x[b], g.x[c], g.x[0]}, by[3] = {g.y[b], g.y[c], g.y[0]};
            // snapped coordinates lie within +-2^29: differences fit int32
            const int OX = tx * TW * 256 + 128, OY = ty * TH * 256 + 128;
            CoverFace cf;
            bool small = true;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const int dx = bx[e] - ax[e], dy = by[e] - ay[e];
                const bool tl = dy < 0 || (dy == 0 && dx > 0);
                const long long E = (long long)dx * (OY - ay[e]) - (long long)dy * (OX - ax[e]) - (tl ? 0 : 1);
                cf.dx[e] = dx;
                cf.dy[e] = dy;
                cf.e0[e] = E;
                cf.thr[e] = (int)max(-2147483647ll, min(2147483647ll, -E));
                small = small && abs(dx) < (1 << 17) && abs(dy) < (1 << 17);
            }
            cf.small = small;
            cf.x0 = g.x[0];
            cf.y0 = g.y[0];
            cf.af = g.af; cf.bf = g.bf; cf.iz0f = g.iz0f;
            cf.f = vf - (unsigned)v * (unsigned)nf;
            s_face[t] = cf;
            s_tex[t] = tex_face(g);
        }
        __syncthreads();
        for (int k = 0; k < nb; ++k) {
            const CoverFace &s = s_face[k];
            // pixel b lies 256 units right of a: E_k(b) = E_k(a) - 256 dy_k
            bool cov0 = true, cov1 = true;
            if (s.small) {
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const int d0 = s.dx[e] * DY - s.dy[e] * DX;
                    cov0 = cov0 && d0 >= s.thr[e];
                    cov1 = cov1 && d0 - s.dy[e] * 256 >= s.thr[e];
                }
            } else {
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const long long E0 = s.e0[e] + (long long)s.dx[e] * DY - (long long)s.dy[e] * DX;
                    const long long E1 = E0 - (long long)s.dy[e] * 256;
                    cov0 = cov0 && E0 >= 0;
                    cov1 = cov1 && E1 >= 0;
                }
            }
            // the 1/z of the face at the pixel centre; the key orders by it
            // (signed: a negative value, possible only through rounding at a
            // sliver, never beats a positive one), then by the lower index
            if (!((cov0 && in[0]) || (cov1 && in[1]))) continue;
            const float Vv = __fmul_rn(__int2float_rn(PY - s.y0), 0.00390625f);
            const float bv = __fmaf_rn(s.bf, Vv, s.iz0f);
            const unsigned long long fkey = ~s.f;
            if (cov0 && in[0]) {
                const float U = __fmul_rn(__int2float_rn(PX - s.x0), 0.00390625f);
                const float iz = __fmaf_rn(s.af, U, bv);
                const long long kk = (long long)(((unsigned long long)__float_as_uint(iz) << 32) | (fkey & 0xFFFFFFFFull));
                if (kk > key[0]) { key[0] = kk; slot[0] = r0 + k; }
            }
            if (cov1 && in[1]) {
                const float U = __fmul_rn(__int2float_rn(PX + 256 - s.x0), 0.00390625f);
                const float iz = __fmaf_rn(s.af, U, bv);
                const long long kk = (long long)(((unsigned long long)__float_as_uint(iz) << 32) | (fkey & 0xFFFFFFFFull));
                if (kk > key[1]) { key[1] = kk; slot[1] = r0 + k; }
            }
        }
    }
    bool hit[2];
    TexFace fs[2];
    float D[2];
    uint32_t fid[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        hit[q] = key[q] != LLONG_MIN;
        fid[q] = ~(uint32_t)((unsigned long long)key[q] & 0xFFFFFFFFull);
        D[q] = hit[q] ? __frcp_rn(__uint_as_float((uint32_t)((unsigned long long)key[q] >> 32))) : INFINITY;
        // the bucket's faces are still staged when it fits one round
        if (hit[q]) fs[q] = fc <= (uint32_t)NT ? s_tex[slot[q]] : tex_face(setup[(long long)v * nf + fid[q]]);
    }
    TexTap tap[2];
#pragma unroll
    for (int q = 0; q < 2; ++q)
        if (hit[q]) tap[q] = tex_tap(fs[q], px + q, py, D[q], tw, th);
    float c[2][3] = {{bg0, bg1, bg2}, {bg0, bg1, bg2}};
    if (hit[0] && hit[1] && tap[0].x0 == tap[1].x0 && tap[0].x1 == tap[1].x1 && tap[0].y0 == tap[1].y0 &&
        tap[0].y1 == tap[1].y1) {
        float tv[4][3];
        texels<F32TEX>(tex, tw, tap[0], tv);
        bilinear_mix<F32TEX>(tap[0], tv, c[0]);
        bilinear_mix<F32TEX>(tap[1], tv, c[1]);
    } else {
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (hit[q]) {
                float tv[4][3];
                texels<F32TEX>(tex, tw, tap[q], tv);
                bilinear_mix<F32TEX>(tap[q], tv, c[q]);
            }
    }
    float m = -INFINITY;   // neutral for the max over in-image pixels
    if (in[0]) m = D[0];
    if (in[1]) m = fmaxf(m, D[1]);
    const int32_t id[2] = {hit[0] ? (int)fid[0] : -1, hit[1] ? (int)fid[1] : -1};
    const float uu[2] = {hit[0] ? tap[0].u : 0.f, hit[1] ? tap[1].u : 0.f};
    const float ww[2] = {hit[0] ? tap[0].w : 0.f, hit[1] ? tap[1].w : 0.f};
    const long long gp = V.pix_off + lp;
    // 8-byte vector stores: both pixels in the image, every plane offset and
    // output pointer even in elements
    const bool vec = in[1] && ((V.pix_off | lp | npx) & 1) == 0 &&
                     (((uintptr_t)tri_id | (uintptr_t)depth | (uintptr_t)rgb | (uintptr_t)uv_out) & 7) == 0;
    if (vec) {
        if (tri_id) *reinterpret_cast<int2 *>(tri_id + gp) = make_int2(id[0], id[1]);
        if (depth) *reinterpret_cast<float2 *>(depth + gp) = make_float2(D[0], D[1]);
        if (rgb) {
            float *o = rgb + 3 * V.pix_off + lp;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                *reinterpret_cast<float2 *>(o + ch * npx) = make_float2(c[0][ch], c[1][ch]);
        }
        if (uv_out) {
            float *o = uv_out + 2 * V.pix_off + lp;
            *reinterpret_cast<float2 *>(o) = make_float2(uu[0], uu[1]);
            *reinterpret_cast<float2 *>(o + npx) = make_float2(ww[0], ww[1]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (!in[q]) continue;
            if (tri_id) tri_id[gp + q] = id[q];
            if (depth) depth[gp + q] = D[q];
            if (rgb) {
                float *o = rgb + 3 * V.pix_off + lp + q;
                o[0] = c[q][0];
                o[npx] = c[q][1];
                o[2 * npx] = c[q][2];
            }
            if (uv_out) {
                float *o = uv_out + 2 * V.pix_off + lp + q;
                o[0] = uu[q];
                o[npx] = ww[q];
            }
        }
    }
    // farthest mesh depth of the tile (+inf if any in-image pixel misses)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) s_max[t >> 5] = m;
    __syncthreads();
    if (t == 0) {
        float r = s_max[0];
        for (int k = 1; k < NT / 32; ++k) r = fmaxf(r, s_max[k]);
        if (tile_max) tile_max[gt] = r;
    }
}

struct RasterWs {
    int2 *sxy;
    double *iz;
    FaceSetup *setup;
    uint32_t *tile_fcnt, *tile_foff, *cursor, *items;
    long long *n_clamped;
    ScanWs scan;
};

RasterWs carve(void *ws, long long mv, long long mf, long long cap, long long tiles, size_t *bytes) {
    WsCarver c(ws);
    RasterWs r;
    r.sxy = c.take<int2>(mv);
    r.iz = c.take<double>(mv);
    r.setup = c.take<FaceSetup>(mf);
    r.tile_fcnt = c.take<uint32_t>(tiles);
    r.tile_foff = c.take<uint32_t>(tiles);
    r.cursor = c.take<uint32_t>(tiles);
    r.items = c.take<uint32_t>(cap);
    r.n_clamped = c.take<long long>(1);
    r.scan.tile_status = c.take<unsigned long long>(scan_tiles(tiles) + 1);
    r.scan.ticket = c.take<unsigned int>(1);
    *bytes = c.off + 256;
    return r;
}

int grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 148 * 16) g = 148 * 16;
    return (int)g;
}

// work items to run: all of them, or none when the capacity was exceeded
__global__ void clamp_items_kernel(const long long *total, long long capacity, long long *n_out) {
    long long t = *total;
    *n_out = t <= capacity ? t : 0;
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" size_t hm_rasterize_mesh_workspace_size(const hm_camera *cams, int32_t n_views,
                                                   int32_t n_verts, int32_t n_faces,
                                                   int64_t item_capacity, const hm_options *opt) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt) || n_verts < 0 || n_faces < 0 || item_capacity < 0)
        return 0;
    size_t bytes = 0;
    carve(nullptr, (long long)n_views * n_verts, (long long)n_views * n_faces, item_capacity,
          vt.total_tiles, &bytes);
    return bytes;
}

extern "C" hm_status hm_rasterize_mesh(const hm_camera *cams, int32_t n_views, const float *verts,
                                       const float *uvs, int32_t n_verts, const int32_t *faces,
                                       int32_t n_faces, const void *tex, int32_t tex_w,
                                       int32_t tex_h, int32_t tex_format, const hm_options *opt,
                                       int32_t *tri_id, float *depth, float *rgb, float *uv,
                                       float *tile_max_depth, int64_t item_capacity,
                                       int64_t *n_items_out, int32_t *d_status, void *ws,
                                       size_t ws_bytes, void *stream) {
    ViewTable vt;
    if (!build_view_table(cams, n_views, opt, &vt)) return HM_ERR_INVALID_ARG;
    if (n_verts < 0 || n_faces < 0) return fail(HM_ERR_INVALID_ARG, "negative mesh size");
    if ((long long)n_views * n_faces >= (1ll << 31) || (long long)n_views * n_verts >= (1ll << 31))
        return fail(HM_ERR_INVALID_ARG, "mesh too large");
    if (tex_format != HM_TEX_RGB8 && tex_format != HM_TEX_RGBF32) return fail(HM_ERR_INVALID_ARG, "tex_format");
    if (tex_w <= 0 || tex_h <= 0 || !tex) return fail(HM_ERR_INVALID_ARG, "texture");
    if (item_capacity < 0 || item_capacity > HM_MAX_PAIRS) return fail(HM_ERR_INVALID_ARG, "item_capacity");
    if (!tri_id || !depth || !tile_max_depth || !n_items_out ||
        (n_faces > 0 && (!verts || !uvs || !faces)))
        return fail(HM_ERR_INVALID_ARG, "null pointer");
    const long long mv = (long long)n_views * n_verts, mf = (long long)n_views * n_faces;
    const long long T = vt.total_tiles;
    size_t need = 0;
    carve(nullptr, mv, mf, item_capacity, T, &need);
    if (!ws || ws_bytes < need) return fail(HM_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    RasterWs r = carve(ws, mv, mf, item_capacity, T, &need);
    cudaError_t e = cudaMemsetAsync(r.tile_fcnt, 0, sizeof(uint32_t) * (size_t)T, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (mv > 0) {
        mesh_vertex_kernel<<<grid_for(mv, 256), 256, 0, s>>>(vt, n_verts, verts, (double)opt->near_mesh, r.sxy, r.iz);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    if (mf > 0) {
        mesh_face_kernel<<<grid_for(mf, 256), 256, 0, s>>>(vt, n_verts, n_faces, faces, uvs, r.sxy, r.iz, r.setup,
                                                           r.tile_fcnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    // per-tile bucket offsets, the item count and the capacity check
    e = launch_scan(r.tile_fcnt, nullptr, r.tile_foff, T, (long long *)n_items_out, item_capacity, d_status,
                    r.scan, s);
    if (e != cudaSuccess) return cuda_status(e);
    clamp_items_kernel<<<1, 1, 0, s>>>((const long long *)n_items_out, item_capacity, r.n_clamped);
    if (mf > 0) {
        e = cudaMemcpyAsync(r.cursor, r.tile_foff, sizeof(uint32_t) * (size_t)T, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_status(e);
        mesh_emit_kernel<<<grid_for(mf, 256), 256, 0, s>>>(vt, n_faces, r.setup, r.n_clamped, r.cursor, r.items);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    const float *bg = opt->bg;
    const bool f32 = tex_format == HM_TEX_RGBF32;
    dim3 tgrid(vt.total_tiles);
#define HM_RASTER(TW, TH)                                                                               \
    do {                                                                                                \
        if (f32)                                                                                        \
            mesh_tile_kernel<TW, TH, true><<<tgrid, TW * TH / 2, 0, s>>>(                               \
                vt, n_faces, r.setup, r.tile_foff, r.tile_fcnt, r.n_clamped, r.items, tex, tex_w, tex_h,   \
                bg[0], bg[1], bg[2], tri_id, depth, rgb, uv, tile_max_depth);                           \
        else                                                                                            \
            mesh_tile_kernel<TW, TH, false><<<tgrid, TW * TH / 2, 0, s>>>(                              \
                vt, n_faces, r.setup, r.tile_foff, r.tile_fcnt, r.n_clamped, r.items, tex, tex_w, tex_h,   \
                bg[0], bg[1], bg[2], tri_id, depth, rgb, uv, tile_max_depth);                           \
    } while (0)
    if (opt->tile_w == 16) HM_RASTER(16, 16);
    else if (opt->tile_w == 32) HM_RASTER(32, 8);
    else HM_RASTER(8, 8);
#undef HM_RASTER
    return cuda_status(cudaGetLastError());
}

#ifdef HM_CHECKED
namespace hm {
HM_CHECKED_READER(mesh)
}  // namespace hm
#endif
