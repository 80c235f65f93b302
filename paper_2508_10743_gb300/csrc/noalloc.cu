// noalloc.cu -- an adjoint of scaling and squaring that allocates nothing.
//
// Some callers cannot allocate device memory at all: a plug-in that only
// receives device buffers from a host application which owns the allocator,
// or a process whose device memory is committed to a fixed budget up front.
// For them cudaMalloc either fails or breaks the owner's accounting, and
// they cannot hand over a workspace either.  darc_exp_backward_noalloc
// therefore keeps its scratch (the two gradient buffers the adjoint
// alternates between) in one file-scope device array of fixed size.  Every
// GPU that loads the library holds that array until the process exits; with
// CUDA's default lazy module loading the driver commits it when the first
// call on a device looks its address up (at load time when
// CUDA_MODULE_LOADING=EAGER).
#include "../../include/darc.h"
#include "kernels.h"

#include <cmath>
#include <mutex>
#include <string>

using namespace darc_impl;

namespace {

// 64 MiB: the adjoint needs 2 x B x 3 x D x H x W floats of scratch, so a
// call may cover at most DARC_NOALLOC_MAX_VOXELS = 2,796,202 voxels summed
// over its batch (one 128^3 volume, or one 160x192x224 volume at half size).
constexpr size_t kScratchFloats = DARC_NOALLOC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float g_scratch[kScratchFloats];

// Device address of g_scratch, looked up once per device with that device
// current.  In host code the name g_scratch is only a host-side stand-in.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
float* g_dev_ptr[kMaxDevices] = {};

int scratch_address(float** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return darc_impl::report_error(DARC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return darc_impl::report_error(DARC_ERR_INTERNAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return darc_impl::report_error(DARC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_dev_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_dev_ptr[dev];
    return DARC_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" int darc_exp_backward_noalloc(const float* v_dev, const float* u_dev, const float* gT_dev,
                                         float* gv_dev, int B, int D, int H, int W, int T, float sign,
                                         void* stream)
{
    if (!v_dev || !u_dev || !gT_dev || !gv_dev) return darc_impl::report_error(DARC_ERR_ARG, "null argument");
    if (B < 1) return darc_impl::report_error(DARC_ERR_ARG, "batch must be >= 1");
    if (D < 2 || H < 2 || W < 2) return darc_impl::report_error(DARC_ERR_SHAPE, "every dimension must be >= 2");
    if (T < 1 || T > 20) return darc_impl::report_error(DARC_ERR_ARG, "T must be 1..20");
    const long long voxels = (long long)B * D * H * W;
    if (voxels > (long long)DARC_NOALLOC_MAX_VOXELS)
        return darc_impl::report_error(
            DARC_ERR_ARG, "darc_exp_backward_noalloc: B*D*H*W = " + std::to_string(voxels) +
                              " exceeds the fixed scratch limit of " + std::to_string(DARC_NOALLOC_MAX_VOXELS) +
                              " voxels; use darc_exp_backward with a workspace");
    if ((long long)div_up(D, VT_Z) * B > 65535)
        return darc_impl::report_error(DARC_ERR_SHAPE, "batch x depth too large for one launch");
    // the last step reads its inputs while it writes gv: gv may replace gT
    // exactly, and must not touch v, u or only part of gT
    const size_t field_bytes = sizeof(float) * 3 * (size_t)voxels;
    if (overlap(gv_dev, field_bytes, v_dev, field_bytes) ||
        overlap(gv_dev, field_bytes, u_dev, field_bytes * (size_t)T) ||
        (gv_dev != gT_dev && overlap(gv_dev, field_bytes, gT_dev, field_bytes)))
        return darc_impl::report_error(DARC_ERR_ARG, "darc_exp_backward_noalloc: gv overlaps v, u or part of gT");
    float* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != DARC_OK) return rc;

    const Vol vol = make_vol(D, H, W);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fb = (size_t)B * 3 * vol.V;
    const float s0 = sign * std::ldexp(1.0f, -T);
    // the steps of darc_exp_backward (g_T -> ... -> g_0) on planar gradients,
    // which fit the scratch array: each buffer cleared before the
    // squaring's adjoint adds into it
    const float* gin = gT_dev;
    for (int t = T - 1; t >= 0; --t) {
        const float* src = (t == 0) ? v_dev : u_dev + (size_t)(t - 1) * fb;
        const float scale = (t == 0) ? s0 : 1.f;
        float* gout;
        if (t == 0)
            gout = (gv_dev == gT_dev && T == 1) ? scratch : gv_dev;
        else
            gout = scratch + (size_t)((T - 1 - t) % 2) * fb;
        cudaError_t e = cudaMemsetAsync(gout, 0, fb * sizeof(float), s);
        if (e == cudaSuccess) e = exp_square_adjoint(src, scale, gin, gout, (t == 0) ? s0 : 1.f, B, vol, s);
        if (e != cudaSuccess) return darc_impl::report_error(DARC_ERR_CUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
        gin = gout;
    }
    if (gv_dev == gT_dev && T == 1) {
        cudaError_t e = cudaMemcpyAsync(gv_dev, scratch, fb * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return darc_impl::report_error(DARC_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
    }
    return DARC_OK;
}
