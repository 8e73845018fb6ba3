// Context: geometry copy, device status word, status read-back.
#include <cmath>
#include <new>

#include "common.cuh"

using namespace utc;

extern "C" int ut_ctx_create(ut_ctx** out, const ut_geometry* geom) {
    if (!out || !geom) return UT_ERR_ARG;
    *out = nullptr;
    const ut_geometry& g = *geom;
    if (g.n_sectors < 1 || g.n_sectors > 4096 || g.strips < 1 || g.strips > 512 || !(g.sector_pitch > 0.f) ||
        !(g.strip_pitch > 0.f))
        return UT_ERR_ARG;
    ut_ctx* c = new (std::nothrow) ut_ctx();
    if (!c) return UT_ERR_ARG;
    c->geom = g;
    c->wait_limit = kSpinLimit;
    c->first_ticket = 0;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess ||
        cudaMalloc(&c->d_status, sizeof(unsigned long long)) != cudaSuccess) {
        delete c;
        return UT_ERR_CUDA;
    }
    if (cudaMallocHost(&c->h_status, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->d_status, 0xFF, sizeof(unsigned long long)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return UT_ERR_CUDA;
    }
    *out = c;
    return UT_OK;
}

extern "C" int ut_ctx_destroy(ut_ctx* c) {
    if (!c) return UT_ERR_ARG;
    int cur = -1;
    const bool swap = cudaGetDevice(&cur) == cudaSuccess && cur != c->device && cudaSetDevice(c->device) == cudaSuccess;
    if (c->d_kmap) cudaFree(c->d_kmap);
    cudaFree(c->d_status);
    cudaFreeHost(c->h_status);
    if (swap) cudaSetDevice(cur);
    delete c;
    return UT_OK;
}

extern "C" int ut_ctx_set_kick_map(ut_ctx* c, int nx, int ny, float tx_max, float ty_max, const float* values) {
    if (!c) return UT_ERR_ARG;
    if (nx == 0) {
        c->kmap_nx = c->kmap_ny = 0;
        return UT_OK;
    }
    if (nx < 2 || nx > 256 || ny < 2 || ny > 256 || !values || !(tx_max > 0.f) || !(ty_max > 0.f) ||
        !std::isfinite(tx_max) || !std::isfinite(ty_max))
        return UT_ERR_ARG;
    float vmax = 0.f;
    for (int i = 0; i < nx * ny; ++i) {
        if (!(values[i] > 0.f) || !std::isfinite(values[i])) return UT_ERR_ARG;
        vmax = values[i] > vmax ? values[i] : vmax;
    }
    // the map lives on the context's device, whichever device is current
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return UT_ERR_CUDA;
    if (cur != c->device && cudaSetDevice(c->device) != cudaSuccess) return UT_ERR_CUDA;
    float* d = nullptr;
    cudaError_t err = cudaMalloc(&d, sizeof(float) * (size_t)nx * ny);
    if (err == cudaSuccess) {
        err = cudaMemcpy(d, values, sizeof(float) * (size_t)nx * ny, cudaMemcpyHostToDevice);
        if (err != cudaSuccess) cudaFree(d);
    }
    if (err == cudaSuccess && c->d_kmap) cudaFree(c->d_kmap);
    if (cur != c->device) cudaSetDevice(cur);
    if (err != cudaSuccess) return UT_ERR_CUDA;
    c->d_kmap = d;
    c->kmap_nx = nx;
    c->kmap_ny = ny;
    c->kmap_tx_max = tx_max;
    c->kmap_ty_max = ty_max;
    c->kmap_max = vmax;
    return UT_OK;
}

extern "C" int ut_ctx_set_wait_limit(ut_ctx* c, long long spins) {
    if (!c) return UT_ERR_ARG;
    c->wait_limit = spins > 0 ? spins : kSpinLimit;
    return UT_OK;
}

extern "C" int ut_ctx_set_first_ticket(ut_ctx* c, int first) {
    if (!c || first < 0) return UT_ERR_ARG;
    c->first_ticket = (unsigned)first;
    return UT_OK;
}

extern "C" int ut_status_reset(ut_ctx* c, void* stream) {
    if (!c) return UT_ERR_ARG;
    return check_cuda(cudaMemsetAsync(c->d_status, 0xFF, sizeof(unsigned long long), static_cast<cudaStream_t>(stream)));
}

extern "C" int ut_status(ut_ctx* c, void* stream, int* code, int64_t* where_a, int64_t* where_b) {
    if (!c || !code) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return UT_ERR_CUDA;
    const unsigned long long k = *c->h_status;
    if (k == ~0ull) {
        *code = UT_OK;
        if (where_a) *where_a = -1;
        if (where_b) *where_b = -1;
        return UT_OK;
    }
    *code = -(int)(k & 0xFF);
    const unsigned long long a = k >> 32, b = (k >> 8) & 0xFFFFFF;
    if (where_a) *where_a = a == 0xFFFFFFFFull ? -1 : (int64_t)a;
    if (where_b) *where_b = b == 0xFFFFFFull ? -1 : (int64_t)b;
    return UT_OK;
}
