// sh.cuh -- real spherical harmonics up to degree 3 in Cartesian form, and
// their gradients.
//
// Basis: the standard real orthonormal SH with the Condon-Shortley phase,
// index l*l + l + m for m = -l..l, evaluated at a unit direction (x,y,z):
//   Y_l^m  = sqrt(2) K_l^m cos(m phi) P_l^m(z),  m > 0
//   Y_l^-m = sqrt(2) K_l^m sin(m phi) P_l^m(z),  m > 0
//   Y_l^0  = K_l^0 P_l(z),   K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
// With sin^m(theta) e^{i m phi} = (x + i y)^m these become polynomials; the
// constants below are the products of K_l^m, sqrt(2) and the Legendre
// coefficients, e.g. Y_1^-1 = -sqrt(3/(4 pi)) y, Y_2^-2 = sqrt(15/(4 pi)) x y,
// Y_3^0 = sqrt(7/(16 pi)) z (2z^2 - 3x^2 - 3y^2).
#pragma once

namespace hm {

constexpr float kSH0 = 0.28209479177387814f;    // sqrt(1/(4 pi))
constexpr float kSH1 = 0.48860251190291992f;    // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;    // sqrt(15/(4 pi))
constexpr float kSH2c = 0.31539156525252005f;   // sqrt(5/(16 pi))
constexpr float kSH2e = 0.54627421529603959f;   // sqrt(15/(16 pi))
constexpr float kSH3a = 0.59004358992664352f;   // sqrt(35/(32 pi))
constexpr float kSH3b = 2.8906114426405538f;    // sqrt(105/(4 pi))
constexpr float kSH3c = 0.45704579946446572f;   // sqrt(21/(32 pi))
constexpr float kSH3d = 0.37317633259011540f;   // sqrt(7/(16 pi))
constexpr float kSH3e = 1.4453057213202769f;    // sqrt(105/(16 pi))

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    Y[0] = kSH0;
    if (DEG >= 1) {
        Y[1] = -kSH1 * y;
        Y[2] = kSH1 * z;
        Y[3] = -kSH1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kSH2a * x * y;
        Y[5] = -kSH2a * y * z;
        Y[6] = kSH2c * (2.f * zz - xx - yy);
        Y[7] = -kSH2a * x * z;
        Y[8] = kSH2e * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kSH3a * y * (3.f * xx - yy);
            Y[10] = kSH3b * x * y * z;
            Y[11] = -kSH3c * y * (4.f * zz - xx - yy);
            Y[12] = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kSH3c * x * (4.f * zz - xx - yy);
            Y[14] = kSH3e * z * (xx - yy);
            Y[15] = -kSH3a * x * (xx - 3.f * yy);
        }
    }
}

// Cartesian gradients dY_k/d(x,y,z) of the polynomials above (before the
// projection onto the sphere's tangent plane, which the caller applies).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float (*G)[3]) {
    G[0][0] = G[0][1] = G[0][2] = 0.f;
    if (DEG >= 1) {
        G[1][0] = 0.f; G[1][1] = -kSH1; G[1][2] = 0.f;
        G[2][0] = 0.f; G[2][1] = 0.f; G[2][2] = kSH1;
        G[3][0] = -kSH1; G[3][1] = 0.f; G[3][2] = 0.f;
    }
    if (DEG >= 2) {
        G[4][0] = kSH2a * y; G[4][1] = kSH2a * x; G[4][2] = 0.f;
        G[5][0] = 0.f; G[5][1] = -kSH2a * z; G[5][2] = -kSH2a * y;
        G[6][0] = -2.f * kSH2c * x; G[6][1] = -2.f * kSH2c * y; G[6][2] = 4.f * kSH2c * z;
        G[7][0] = -kSH2a * z; G[7][1] = 0.f; G[7][2] = -kSH2a * x;
        G[8][0] = 2.f * kSH2e * x; G[8][1] = -2.f * kSH2e * y; G[8][2] = 0.f;
        if (DEG >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            G[9][0] = -6.f * kSH3a * x * y; G[9][1] = -3.f * kSH3a * (xx - yy); G[9][2] = 0.f;
            G[10][0] = kSH3b * y * z; G[10][1] = kSH3b * x * z; G[10][2] = kSH3b * x * y;
            G[11][0] = 2.f * kSH3c * x * y; G[11][1] = -kSH3c * (4.f * zz - xx - 3.f * yy); G[11][2] = -8.f * kSH3c * y * z;
            G[12][0] = -6.f * kSH3d * x * z; G[12][1] = -6.f * kSH3d * y * z; G[12][2] = kSH3d * (6.f * zz - 3.f * xx - 3.f * yy);
            G[13][0] = -kSH3c * (4.f * zz - 3.f * xx - yy); G[13][1] = 2.f * kSH3c * x * y; G[13][2] = -8.f * kSH3c * x * z;
            G[14][0] = 2.f * kSH3e * x * z; G[14][1] = -2.f * kSH3e * y * z; G[14][2] = kSH3e * (xx - yy);
            G[15][0] = -3.f * kSH3a * (xx - yy); G[15][1] = 6.f * kSH3a * x * y; G[15][2] = 0.f;
        }
    }
}

// sum_k w[k] dY_k/d(x,y,z): the Cartesian gradient of the weighted sum of
// the polynomials above (the same derivatives as sh_basis_grad, accumulated
// term by term so that no K x 3 table is held)
template <int DEG>
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, const float *w, float &gx,
                                            float &gy, float &gz) {
    gx = gy = gz = 0.f;
    if (DEG >= 1) {
        gx = -kSH1 * w[3];
        gy = -kSH1 * w[1];
        gz = kSH1 * w[2];
    }
    if (DEG >= 2) {
        gx += kSH2a * (w[4] * y - w[7] * z) + 2.f * x * (kSH2e * w[8] - kSH2c * w[6]);
        gy += kSH2a * (w[4] * x - w[5] * z) - 2.f * y * (kSH2c * w[6] + kSH2e * w[8]);
        gz += 4.f * kSH2c * w[6] * z - kSH2a * (w[5] * y + w[7] * x);
        if (DEG >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            const float xy = x * y, xz = x * z, yz = y * z;
            // Y9 = -a y (3xx - yy)
            gx += w[9] * (-6.f * kSH3a * xy);
            gy += w[9] * (-3.f * kSH3a * (xx - yy));
            // Y10 = b x y z
            gx += w[10] * (kSH3b * yz);
            gy += w[10] * (kSH3b * xz);
            gz += w[10] * (kSH3b * xy);
            // Y11 = -c y (4zz - xx - yy)
            gx += w[11] * (2.f * kSH3c * xy);
            gy += w[11] * (-kSH3c * (4.f * zz - xx - 3.f * yy));
            gz += w[11] * (-8.f * kSH3c * yz);
            // Y12 = d z (2zz - 3xx - 3yy)
            gx += w[12] * (-6.f * kSH3d * xz);
            gy += w[12] * (-6.f * kSH3d * yz);
            gz += w[12] * (kSH3d * (6.f * zz - 3.f * xx - 3.f * yy));
            // Y13 = -c x (4zz - xx - yy)
            gx += w[13] * (-kSH3c * (4.f * zz - 3.f * xx - yy));
            gy += w[13] * (2.f * kSH3c * xy);
            gz += w[13] * (-8.f * kSH3c * xz);
            // Y14 = e z (xx - yy)
            gx += w[14] * (2.f * kSH3e * xz);
            gy += w[14] * (-2.f * kSH3e * yz);
            gz += w[14] * (kSH3e * (xx - yy));
            // Y15 = -a x (xx - 3yy)
            gx += w[15] * (-3.f * kSH3a * (xx - yy));
            gy += w[15] * (6.f * kSH3a * xy);
        }
    }
}

}  // namespace hm
