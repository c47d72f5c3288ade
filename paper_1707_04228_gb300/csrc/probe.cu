// FP64 FMA throughput probe: the denominator of the FP64-bound kernels'
// roofline fractions (the matrix-free K u and the FP64 local sweeps).
//
// Every thread runs CHAINS independent chains of dependent FP64 FMAs
// (a <- a * b + c), enough chains per warp to cover the FMA latency, on a
// grid of BLOCKS_PER_SM blocks per SM; nothing is read from or written to
// memory inside the loop.  The result is folded into one value that is
// written only if it equals an impossible sentinel, which keeps the compiler
// from removing the work without adding memory traffic.
#include "gl_internal.h"

namespace gl {

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_fp64_probe(int iters, double b, double c, double *sink) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == -12345.678) *sink = s;
}

}  // namespace

// Runs the probe on the current device: `reps` launches of `iters` iterations
// after one warm-up launch; returns FMA flops per second (2 per FMA).
double fp64_probe(int iters, int reps, int *n_sm, double *ms_out) {
    int dev = 0, sms = 0;
    GL_CUDA(cudaGetDevice(&dev));
    GL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DBuf<double> sink;
    sink.alloc(1);
    cudaStream_t s = nullptr;
    GL_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GL_CUDA(cudaEventCreate(&e0));
    GL_CUDA(cudaEventCreate(&e1));
    const int blocks = sms * PROBE_BLOCKS_PER_SM;
    // b slightly below 1 keeps the chains bounded; the values never matter
    k_fp64_probe<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999999, 1e-7, sink.p);
    GL_CUDA(cudaGetLastError());
    GL_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) k_fp64_probe<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999999, 1e-7, sink.p);
    GL_CUDA(cudaGetLastError());
    GL_CUDA(cudaEventRecord(e1, s));
    GL_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    const double fmas = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)iters * reps;
    if (n_sm) *n_sm = sms;
    if (ms_out) *ms_out = ms;
    return 2.0 * fmas / (ms / 1e3);
}

}  // namespace gl
