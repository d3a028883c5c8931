// adam.cu -- the Adam update (Kingma and Ba, 2015) for optimised buffers such
// as the texture map of the texture-only optimisation (Sec. 3.3): per element
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - lr (m / c1) / (sqrt(v / c2) + eps),  c1 = 1 - b1^t, c2 = 1 - b2^t.
// Memory-bound: 4 floats read, 3 written per element, four at a time.
#include <math.h>

#include "hm_host.h"

namespace hm {

namespace {

__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                      float rc1, float rc2, float eps) {
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p -= lr * (m * rc1) / (sqrtf(v * rc2) + eps);
}

// rc = (1 / (1 - b1^t), 1 / (1 - b2^t)) from the host (rc_dev null) or from
// device memory (a step captured in a CUDA graph); a nonzero *status (an
// earlier stage reported an error) skips the update
__global__ void __launch_bounds__(256)
adam_kernel(long long n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
            float *__restrict__ v, float lr, float b1, float b2, float rc1, float rc2, float eps, bool vec4,
            const float *__restrict__ rc_dev, const int32_t *__restrict__ status) {
    if (status && *status) return;
    if (rc_dev) {
        rc1 = rc_dev[0];
        rc2 = rc_dev[1];
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tail = 0;
    if (vec4) {
        const long long n4 = n >> 2;
        for (long long i = tid; i < n4; i += stride) {
            float4 P = reinterpret_cast<float4 *>(p)[i], M = reinterpret_cast<float4 *>(m)[i];
            float4 Vv = reinterpret_cast<float4 *>(v)[i];
            const float4 G = reinterpret_cast<const float4 *>(g)[i];
            adam1(P.x, G.x, M.x, Vv.x, lr, b1, b2, rc1, rc2, eps);
            adam1(P.y, G.y, M.y, Vv.y, lr, b1, b2, rc1, rc2, eps);
            adam1(P.z, G.z, M.z, Vv.z, lr, b1, b2, rc1, rc2, eps);
            adam1(P.w, G.w, M.w, Vv.w, lr, b1, b2, rc1, rc2, eps);
            reinterpret_cast<float4 *>(p)[i] = P;
            reinterpret_cast<float4 *>(m)[i] = M;
            reinterpret_cast<float4 *>(v)[i] = Vv;
        }
        tail = n4 << 2;
    }
    for (long long i = tail + tid; i < n; i += stride) adam1(p[i], g[i], m[i], v[i], lr, b1, b2, rc1, rc2, eps);
}

}  // namespace

}  // namespace hm

using namespace hm;

static hm_status launch_adam(float *param, const float *grad, float *m, float *v, int64_t n, float lr, float beta1,
                             float beta2, float eps, float rc1, float rc2, const float *d_rc, const int32_t *d_status,
                             void *stream) {
    const bool vec4 = (((uintptr_t)param | (uintptr_t)grad | (uintptr_t)m | (uintptr_t)v) & 15) == 0;
    const long long work = vec4 ? (n >> 2) + 1 : n;
    const int grid = (int)((work + 255) / 256 < 148 * 8 ? (work + 255) / 256 : 148 * 8);
    adam_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(n, param, grad, m, v, lr, beta1, beta2, rc1, rc2, eps, vec4,
                                                        d_rc, d_status);
    return cuda_status(cudaGetLastError());
}

extern "C" hm_status hm_adam_update(float *param, const float *grad, float *m, float *v, int64_t n, float lr,
                                    float beta1, float beta2, float eps, int32_t step, void *stream) {
    if (n < 0 || step < 1) return fail(HM_ERR_INVALID_ARG, "n < 0 or step < 1");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f) || !(lr >= 0.f))
        return fail(HM_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    if (n == 0) return HM_OK;
    if (!param || !grad || !m || !v) return fail(HM_ERR_INVALID_ARG, "null pointer");
    const float rc1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
    const float rc2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
    return launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, rc1, rc2, nullptr, nullptr, stream);
}

extern "C" hm_status hm_adam_update_dev(float *param, const float *grad, float *m, float *v, int64_t n, float lr,
                                        float beta1, float beta2, float eps, const float *d_rc,
                                        const int32_t *d_status, void *stream) {
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f) || !(lr >= 0.f))
        return fail(HM_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    if (n == 0) return HM_OK;
    if (!param || !grad || !m || !v || !d_rc) return fail(HM_ERR_INVALID_ARG, "null pointer");
    return launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, 1.f, 1.f, d_rc, d_status, stream);
}
