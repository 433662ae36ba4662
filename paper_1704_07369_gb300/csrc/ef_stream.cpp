// ef_stream.cpp -- batches that live in host memory, streamed through the GPU: the batch is cut
// into contiguous chunks of cells, each with its own batched plan and CUDA stream, so that the
// upload of one chunk, the collision step of another and the download of a third overlap (one
// copy engine each way, the SMs in between).  Built only on the public entry points of ef.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "ef.h"
#include "ef_launch.h"

struct ef_stream_plan_s {
    int d = 3;
    size_t el = 4;
    int64_t ncells = 0;
    struct Chunk {
        ef_plan_t plan = nullptr;
        int64_t c0 = 0, nc = 0;        // first cell and cell count
        int64_t e0 = 0, ne = 0;        // first element and element count
        cudaStream_t s = nullptr;        // one of the compute streams (not owned)
        cudaEvent_t up = nullptr;        // the chunk's upload is done
        cudaEvent_t done = nullptr;      // the chunk's steps (and diagnostics copies) are done
    };
    std::vector<Chunk> chunks;
    // a three-stage pipeline: every upload on one stream (the host-to-device copies run back to
    // back), the steps on a few compute streams (at most kComputeStreams chunks in flight, so that
    // their small launches do not crowd each other off the SMs), every download on one stream
    cudaStream_t up_s = nullptr, down_s = nullptr;
    std::vector<cudaStream_t> comp;
    cudaEvent_t down_done = nullptr;
    void *F_dev = nullptr;
    double *diag_dev = nullptr;        // one step's diagnostics of the whole batch (made at create)
    cudaEvent_t fork = nullptr;
    int device = 0;
};

namespace {

constexpr int kComputeStreams = 4;

ef_status sp_fail(ef_status s, const std::string &m)
{
    ef::set_last_error(m.c_str());
    return s;
}

ef_status sp_cuda(cudaError_t e, const char *what)
{
    const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    ef::set_last_error(m.c_str());
    return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
}

void sp_free(ef_stream_plan_s *sp)
{
    if (!sp) return;
    for (auto &c : sp->chunks) {
        if (c.plan) ef_plan_destroy(c.plan);
        if (c.up) cudaEventDestroy(c.up);
        if (c.done) cudaEventDestroy(c.done);
    }
    for (cudaStream_t q : sp->comp)
        if (q) cudaStreamDestroy(q);
    if (sp->up_s) cudaStreamDestroy(sp->up_s);
    if (sp->down_s) cudaStreamDestroy(sp->down_s);
    if (sp->down_done) cudaEventDestroy(sp->down_done);
    if (sp->fork) cudaEventDestroy(sp->fork);
    cudaFree(sp->F_dev);
    cudaFree(sp->diag_dev);
    delete sp;
}

}  // namespace

extern "C" {

ef_status ef_stream_plan_create(int d, int64_t ncells, const int *N_host, double L, ef_kernel kernel, int R,
                                ef_precision prec, int nchunks, ef_stream_plan_t *out)
{
    if (!out) return sp_fail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (ncells <= 0 || !N_host) return sp_fail(EF_ERR_INVALID_ARG, "stream plan needs ncells > 0 and N_host");
    if (nchunks < 1) return sp_fail(EF_ERR_INVALID_ARG, "nchunks must be >= 1");
    if (d != 2 && d != 3) return sp_fail(EF_ERR_INVALID_ARG, "d must be 2 or 3");
    if (nchunks > ncells) nchunks = (int)ncells;
    // contiguous chunks of about equal work (N^d log N^d per cell)
    std::vector<double> cost(ncells);
    double total = 0.0;
    for (int64_t c = 0; c < ncells; ++c) {
        if (N_host[c] < 2) return sp_fail(EF_ERR_INVALID_ARG, "cell size N must be >= 2");
        const double m = std::pow((double)N_host[c], d);
        cost[c] = m * std::log2(m);
        total += cost[c];
    }
    ef_stream_plan_s *sp = new ef_stream_plan_s();
    sp->d = d;
    sp->el = prec == EF_PREC_F32 ? 4 : 8;
    sp->ncells = ncells;
    cudaError_t e = cudaGetDevice(&sp->device);
    if (e != cudaSuccess) { sp_free(sp); return sp_cuda(e, "cudaGetDevice"); }
    int64_t c = 0, elem = 0;
    double acc = 0.0;
    for (int k = 0; k < nchunks && c < ncells; ++k) {
        ef_stream_plan_s::Chunk ch;
        ch.c0 = c;
        ch.e0 = elem;
        const double target = total * (k + 1) / nchunks;
        const int64_t left = nchunks - k - 1;          // keep at least one cell per later chunk
        while (c < ncells && (c == ch.c0 || (acc + cost[c] <= target + 0.5 * cost[c] && ncells - c > left))) {
            acc += cost[c];
            elem += d == 3 ? (int64_t)N_host[c] * N_host[c] * N_host[c] : (int64_t)N_host[c] * N_host[c];
            ++c;
        }
        if (k == nchunks - 1) {                       // the last chunk takes the rest
            while (c < ncells) {
                elem += d == 3 ? (int64_t)N_host[c] * N_host[c] * N_host[c] : (int64_t)N_host[c] * N_host[c];
                ++c;
            }
        }
        ch.nc = c - ch.c0;
        ch.ne = elem - ch.e0;
        ef_status st = ef_plan_create_batched(d, ch.nc, N_host + ch.c0, L, kernel, R, prec, &ch.plan);
        if (st != EF_OK) { sp_free(sp); return st; }
        if ((int)sp->comp.size() < kComputeStreams) {
            cudaStream_t q = nullptr;
            e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
            sp->comp.push_back(q);
        }
        ch.s = sp->comp[sp->chunks.size() % sp->comp.size()];
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ch.up, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ch.done, cudaEventDisableTiming);
        sp->chunks.push_back(ch);
        if (e != cudaSuccess) { sp_free(sp); return sp_cuda(e, "chunk stream"); }
    }
    e = cudaEventCreateWithFlags(&sp->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sp->down_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sp->up_s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sp->down_s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sp->F_dev, (size_t)elem * sp->el);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sp->diag_dev, (size_t)ncells * EF_DIAG_STRIDE * sizeof(double));
    if (e != cudaSuccess) { sp_free(sp); return sp_cuda(e, "stream plan buffers"); }
    *out = sp;
    return EF_OK;
}

ef_status ef_stream_plan_destroy(ef_stream_plan_t sp)
{
    if (!sp) return sp_fail(EF_ERR_INVALID_ARG, "null stream plan");
    int cur = -1;
    const bool had = cudaGetDevice(&cur) == cudaSuccess;
    const int dev = sp->device;
    cudaSetDevice(dev);                 // free on the plan's device, then restore the caller's
    cudaDeviceSynchronize();
    sp_free(sp);
    if (had && cur != dev) cudaSetDevice(cur);
    return EF_OK;
}

ef_status ef_stream_plan_info(ef_stream_plan_t sp, int64_t info[4])
{
    if (!sp || !info) return sp_fail(EF_ERR_INVALID_ARG, "null stream plan or info");
    int64_t elems = 0;
    for (const auto &c : sp->chunks) elems += c.ne;
    info[0] = sp->ncells;
    info[1] = (int64_t)sp->chunks.size();
    info[2] = elems;
    info[3] = (int64_t)sp->el;
    return EF_OK;
}

ef_status ef_stream_euler_step(ef_stream_plan_t sp, void *F_host, double dt, int nsteps, double *diag_host,
                               ef_stream_t stream)
{
    if (!sp) return sp_fail(EF_ERR_INVALID_ARG, "null stream plan");
    if (nsteps < 0 || !std::isfinite(dt)) return sp_fail(EF_ERR_INVALID_ARG, "negative nsteps or non-finite dt");
    if (nsteps == 0) return EF_OK;
    if (!F_host) return sp_fail(EF_ERR_INVALID_ARG, "null F_host");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev != sp->device) return sp_fail(EF_ERR_INVALID_ARG, "the stream plan's device is not current");
    cudaStream_t cs = (cudaStream_t)stream;
    e = cudaEventRecord(sp->fork, cs);
    if (e != cudaSuccess) return sp_cuda(e, "fork");
    unsigned char *Fh = static_cast<unsigned char *>(F_host);
    unsigned char *Fd = static_cast<unsigned char *>(sp->F_dev);
    const size_t row = EF_DIAG_STRIDE * sizeof(double);
    ef_status st = EF_OK;
    // every stream of the plan waits for the caller's prior work; the uploads also wait for the
    // previous call's downloads (the device buffer is reused, whatever stream that call was on)
    e = cudaStreamWaitEvent(sp->up_s, sp->fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sp->up_s, sp->down_done, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sp->down_s, sp->fork, 0);
    for (size_t j = 0; e == cudaSuccess && j < sp->comp.size(); ++j) e = cudaStreamWaitEvent(sp->comp[j], sp->fork, 0);
    if (e != cudaSuccess) return sp_cuda(e, "fork wait");
    for (auto &c : sp->chunks) {
        // upload (one stream: the copies run back to back), steps (the chunk's compute stream, after
        // its upload), download (one stream, after the chunk's steps)
        e = cudaMemcpyAsync(Fd + c.e0 * sp->el, Fh + c.e0 * sp->el, c.ne * sp->el, cudaMemcpyHostToDevice, sp->up_s);
        if (e == cudaSuccess) e = cudaEventRecord(c.up, sp->up_s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c.s, c.up, 0);
        if (e != cudaSuccess) { st = sp_cuda(e, "upload"); break; }
        // one step at a time: the chunk's slice of the one-step diagnostics buffer is copied out
        // on the chunk's stream before the next step overwrites it
        double *dd = diag_host ? sp->diag_dev + (size_t)c.c0 * EF_DIAG_STRIDE : nullptr;
        for (int k = 0; k < nsteps && st == EF_OK; ++k) {
            st = ef_euler_step(c.plan, Fd + c.e0 * sp->el, dt, 1, dd, c.nc, (ef_stream_t)c.s);
            if (st == EF_OK && diag_host) {
                e = cudaMemcpyAsync(diag_host + ((size_t)k * sp->ncells + c.c0) * EF_DIAG_STRIDE, dd, c.nc * row,
                                    cudaMemcpyDeviceToHost, c.s);
                if (e != cudaSuccess) st = sp_cuda(e, "diagnostics download");
            }
        }
        if (st != EF_OK) break;
        e = cudaEventRecord(c.done, c.s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sp->down_s, c.done, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Fh + c.e0 * sp->el, Fd + c.e0 * sp->el, c.ne * sp->el, cudaMemcpyDeviceToHost, sp->down_s);
        if (e != cudaSuccess) { st = sp_cuda(e, "download"); break; }
    }
    // join every stream of the plan into the caller's stream, on success and on an error part way
    // (so that F_host and diag_host are free for reuse once `stream` has completed); the events
    // are recorded after all work enqueued so far on each stream
    e = cudaEventRecord(sp->down_done, sp->up_s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, sp->down_done, 0);
    if (e != cudaSuccess && st == EF_OK) st = sp_cuda(e, "join");
    for (size_t j = 0; j < sp->comp.size(); ++j) {
        e = cudaEventRecord(sp->chunks[j].done, sp->comp[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, sp->chunks[j].done, 0);
        if (e != cudaSuccess && st == EF_OK) st = sp_cuda(e, "join");
    }
    e = cudaEventRecord(sp->down_done, sp->down_s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, sp->down_done, 0);
    if (e != cudaSuccess && st == EF_OK) st = sp_cuda(e, "join");
    return st;
}

ef_status ef_stream_plan_status(ef_stream_plan_t sp, int sync, int reset)
{
    if (!sp) return sp_fail(EF_ERR_INVALID_ARG, "null stream plan");
    ef_status first = EF_OK;
    for (auto &c : sp->chunks) {
        const ef_status st = ef_plan_status(c.plan, sync, reset);
        if (first == EF_OK && st != EF_OK) first = st;
    }
    return first;
}

}  // extern "C"
