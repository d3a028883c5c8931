// train.cu -- the element-wise pieces of the joint optimisation step around
// the renderer (Sec. 3.4), for a step that runs as one CUDA graph:
//  * the 3DGS parameterisation: scales = exp(log-scales), opacity =
//    sigmoid(logit), and the chain rule back to the raw parameters;
//  * the Adam step counter and its bias corrections kept in device memory.
#include <math.h>

#include "hm_host.h"

namespace hm {

namespace {

__global__ void __launch_bounds__(256)
activate_kernel(long long n, const float *__restrict__ log_s, const float *__restrict__ logit,
                float *__restrict__ scales, float *__restrict__ opacity) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += stride) {
        scales[i] = expf(log_s[i]);
        if (i < n) opacity[i] = 1.f / (1.f + expf(-logit[i]));
    }
}

__global__ void __launch_bounds__(256)
activate_bwd_kernel(long long n, const float *__restrict__ scales, const float *__restrict__ opacity,
                    const float *__restrict__ d_scales, const float *__restrict__ d_opacity,
                    float *__restrict__ d_log_s, float *__restrict__ d_logit) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += stride) {
        d_log_s[i] = d_scales[i] * scales[i];                         // d exp(x) = exp(x)
        if (i < n) d_logit[i] = d_opacity[i] * (opacity[i] * (1.f - opacity[i]));   // d sigmoid = s (1 - s)
    }
}

// ++t and the bias corrections 1 / (1 - b^t), unless *status reports an error
__global__ void adam_advance_kernel(int32_t *step, float b1, float b2, float *rc, const int32_t *status) {
    if (status && *status) return;
    const int t = ++*step;
    rc[0] = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
    rc[1] = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
}

int grid_of(long long work) {
    const long long g = (work + 255) / 256;
    return (int)(g < 148 * 8 ? (g > 0 ? g : 1) : 148 * 8);
}

}  // namespace

}  // namespace hm

using namespace hm;

extern "C" hm_status hm_activate(int64_t n, const float *log_scales, const float *logit, float *scales,
                                 float *opacity, void *stream) {
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return HM_OK;
    if (!log_scales || !logit || !scales || !opacity) return fail(HM_ERR_INVALID_ARG, "null pointer");
    activate_kernel<<<grid_of(3 * n), 256, 0, (cudaStream_t)stream>>>(n, log_scales, logit, scales, opacity);
    return cuda_status(cudaGetLastError());
}

extern "C" hm_status hm_activate_backward(int64_t n, const float *scales, const float *opacity,
                                          const float *d_scales, const float *d_opacity, float *d_log_scales,
                                          float *d_logit, void *stream) {
    if (n < 0) return fail(HM_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return HM_OK;
    if (!scales || !opacity || !d_scales || !d_opacity || !d_log_scales || !d_logit)
        return fail(HM_ERR_INVALID_ARG, "null pointer");
    activate_bwd_kernel<<<grid_of(3 * n), 256, 0, (cudaStream_t)stream>>>(n, scales, opacity, d_scales, d_opacity,
                                                                         d_log_scales, d_logit);
    return cuda_status(cudaGetLastError());
}

extern "C" hm_status hm_adam_advance(int32_t *d_step, float beta1, float beta2, float *d_rc, const int32_t *d_status,
                                     void *stream) {
    if (!d_step || !d_rc) return fail(HM_ERR_INVALID_ARG, "null pointer");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
        return fail(HM_ERR_INVALID_ARG, "betas out of range");
    adam_advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_step, beta1, beta2, d_rc, d_status);
    return cuda_status(cudaGetLastError());
}
