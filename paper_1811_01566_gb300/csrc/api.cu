// Status strings and version of the libwf C ABI.
#include "common.cuh"

extern "C" const char* wf_status_string(wf_status s) {
    switch (s) {
        case WF_OK: return "WF_OK";
        case WF_ERR_INVALID_ARG: return "WF_ERR_INVALID_ARG: invalid argument";
        case WF_ERR_UNSUPPORTED: return "WF_ERR_UNSUPPORTED: outside the supported limits";
        case WF_ERR_CUDA: return "WF_ERR_CUDA: CUDA launch or runtime error";
        case WF_ERR_WORKSPACE: return "WF_ERR_WORKSPACE: workspace missing or too small";
        case WF_ERR_INTERNAL: return "WF_ERR_INTERNAL: kernel recorded an internal inconsistency";
    }
    return "unknown wf_status";
}

extern "C" int32_t wf_version(void) { return 100; }

extern "C" wf_status wf_stream_create(wf_stream* out) {
    if (!out) return WF_ERR_INVALID_ARG;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        *out = nullptr;
        return WF_ERR_CUDA;
    }
    *out = reinterpret_cast<wf_stream>(s);
    return WF_OK;
}

extern "C" wf_status wf_stream_destroy(wf_stream stream) {
    if (!stream) return WF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e1 = cudaStreamSynchronize(s);
    const cudaError_t e2 = cudaStreamDestroy(s);
    return e1 == cudaSuccess && e2 == cudaSuccess ? WF_OK : WF_ERR_CUDA;
}
