// Batched independent acquisitions (many autofocus problems in one job).
//
// A batch owns one plan and one non-blocking stream per member, a capture
// stream and the events that fork member streams from a stream and join them
// back.  af_batch_iterate runs one af_iterate of every member concurrently;
// af_batch_capture records n iterations of every member into one CUDA graph
// (stream capture: every af_* call of an iteration only enqueues kernels and
// async memsets on its plan's stream, and the Adam step index is a launch
// argument), and af_batch_launch replays the whole job with one graph launch.
// This file sequences calls; every step of the computation is a library kernel.
#include <vector>

#include "af_internal.cuh"

struct af_batch_s {
    int n = 0;
    std::vector<af_plan_t> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;      // member k finished its work of the current issue
    cudaStream_t caller = nullptr;      // the caller's stream (may be the legacy default)
    cudaStream_t cap = nullptr;         // capture / launch stream of the graph
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

af_status batch_cuda(const char *what, cudaError_t e)
{
    return af_set_error(AF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BT_CHECK(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return batch_cuda(#call, e_);    \
    } while (0)

struct BatchArgs {
    const void *const *iq;
    const float *const *scale;
    float *const *s, *const *grad, *const *m, *const *v, *const *loss;
};

af_status check_args(const af_batch_s *b, const BatchArgs &a)
{
    if (!a.iq || !a.s || !a.grad || !a.m || !a.v || !a.loss)
        return af_set_error(AF_ERR_ARG, "af_batch: a pointer array is NULL");
    for (int k = 0; k < b->n; ++k)
        if (!a.iq[k] || !a.s[k] || !a.grad[k] || !a.m[k] || !a.v[k] || !a.loss[k])
            return af_set_error(AF_ERR_ARG, "af_batch: member %d has a NULL device pointer", k);
    return AF_OK;
}

// one iteration of every member, forked from `origin` and joined back to it;
// when a member fails, the members issued so far (the failing one included,
// which may have enqueued part of its work) are still joined, so later work on
// `origin` stays ordered after everything this call enqueued
af_status issue(af_batch_s *b, cudaStream_t origin, const BatchArgs &a, int step)
{
    BT_CHECK(cudaEventRecord(b->fork, origin));
    af_status st = AF_OK;
    int issued = 0;
    for (int k = 0; k < b->n && st == AF_OK; ++k) {
        BT_CHECK(cudaStreamWaitEvent(b->streams[k], b->fork, 0));
        st = af_iterate(b->plans[k], a.iq[k], a.scale ? a.scale[k] : nullptr, a.s[k], a.grad[k], a.m[k], a.v[k],
                        step, a.loss[k]);
        BT_CHECK(cudaEventRecord(b->done[k], b->streams[k]));
        issued = k + 1;
    }
    for (int k = 0; k < issued; ++k) BT_CHECK(cudaStreamWaitEvent(origin, b->done[k], 0));
    return st;
}

void release(af_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (af_plan_t p : b->plans)
        if (p) af_destroy(p);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // namespace

extern "C" af_status af_batch_plan(int n, const af_config *const *cfgs, void *stream, af_batch_t *out)
{
    if (!out) return af_set_error(AF_ERR_ARG, "af_batch_plan: out is NULL");
    *out = nullptr;
    if (n < 1 || !cfgs) return af_set_error(AF_ERR_ARG, "af_batch_plan: need n >= 1 configurations");
    for (int k = 0; k < n; ++k) {
        if (!cfgs[k]) return af_set_error(AF_ERR_ARG, "af_batch_plan: configuration %d is NULL", k);
        const af_status st = af_check_config(cfgs[k]);
        if (st != AF_OK) return st;
    }
    af_batch_s *b = new af_batch_s;
    b->n = n;
    b->caller = (cudaStream_t)stream;
    b->plans.assign(n, nullptr);
    b->streams.assign(n, nullptr);
    b->done.assign(n, nullptr);
    auto bail = [&](af_status st) { release(b); return st; };
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return bail(batch_cuda("af_batch_plan: streams / events", e));
    for (int k = 0; k < n; ++k) {
        const af_status st = af_plan(cfgs[k], b->streams[k], &b->plans[k]);
        if (st != AF_OK) return bail(st);
    }
    *out = b;
    return af_set_error(AF_OK, "");
}

extern "C" af_status af_batch_plan_of(af_batch_t b, int k, af_plan_t *out)
{
    if (!b || !out) return af_set_error(AF_ERR_ARG, "af_batch_plan_of: NULL argument");
    if (k < 0 || k >= b->n) return af_set_error(AF_ERR_ARG, "af_batch_plan_of: member %d of %d", k, b->n);
    *out = b->plans[k];
    return af_set_error(AF_OK, "");
}

extern "C" af_status af_batch_iterate(af_batch_t b, const void *const *d_iq, const float *const *d_iq_scale,
                                      float *const *d_s, float *const *d_grad, float *const *d_m,
                                      float *const *d_v, int step, float *const *d_loss)
{
    if (!b) return af_set_error(AF_ERR_ARG, "af_batch_iterate: batch is NULL");
    const BatchArgs a{d_iq, d_iq_scale, d_s, d_grad, d_m, d_v, d_loss};
    af_status st = check_args(b, a);
    if (st != AF_OK) return st;
    st = issue(b, b->caller, a, step);
    return st == AF_OK ? af_set_error(AF_OK, "") : st;
}

extern "C" af_status af_batch_capture(af_batch_t b, const void *const *d_iq, const float *const *d_iq_scale,
                                      float *const *d_s, float *const *d_grad, float *const *d_m,
                                      float *const *d_v, float *const *d_loss, int first_step, int n_iter)
{
    if (!b) return af_set_error(AF_ERR_ARG, "af_batch_capture: batch is NULL");
    if (first_step < 1 || n_iter < 1)
        return af_set_error(AF_ERR_ARG, "af_batch_capture: first_step %d, n_iter %d", first_step, n_iter);
    const BatchArgs a{d_iq, d_iq_scale, d_s, d_grad, d_m, d_v, d_loss};
    af_status st = check_args(b, a);
    if (st != AF_OK) return st;
    for (int k = 0; k < b->n; ++k)
        if (b->plans[k]->timing) return af_set_error(AF_ERR_STATE, "af_batch_capture: stage timing is on (member %d)", k);
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    // the capture stream starts after the caller's earlier work (outside the capture)
    BT_CHECK(cudaEventRecord(b->ev_in, b->caller));
    BT_CHECK(cudaStreamWaitEvent(b->cap, b->ev_in, 0));
    BT_CHECK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < n_iter && st == AF_OK; ++it) st = issue(b, b->cap, a, first_step + it);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (st != AF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return batch_cuda("af_batch_capture: cudaStreamEndCapture", e);
    b->graph = graph;
    BT_CHECK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return af_set_error(AF_OK, "");
}

extern "C" af_status af_batch_launch(af_batch_t b)
{
    if (!b) return af_set_error(AF_ERR_ARG, "af_batch_launch: batch is NULL");
    if (!b->exec) return af_set_error(AF_ERR_STATE, "af_batch_launch: nothing captured");
    BT_CHECK(cudaEventRecord(b->ev_in, b->caller));
    BT_CHECK(cudaStreamWaitEvent(b->cap, b->ev_in, 0));
    BT_CHECK(cudaGraphLaunch(b->exec, b->cap));
    BT_CHECK(cudaEventRecord(b->ev_out, b->cap));
    BT_CHECK(cudaStreamWaitEvent(b->caller, b->ev_out, 0));
    return af_set_error(AF_OK, "");
}

extern "C" af_status af_batch_destroy(af_batch_t b)
{
    if (b) release(b);
    return AF_OK;
}
