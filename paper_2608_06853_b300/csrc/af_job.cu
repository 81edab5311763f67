// Autofocus jobs from host memory: the upload of one acquisition's channel
// data and initial map, N_i iterations of the method (Sec. III-A, Table II)
// and the read back of the final map and loss, as one call.
//
// A plan that runs jobs keeps two device buffers for channel data, the
// iteration state (map, gradient, Adam moments, loss) and a copy stream.  A
// submitted job enqueues its upload on the copy stream, into the buffer the
// job before last used, and its iterations on the plan's stream, and returns;
// so the next job's upload runs under the current job's iterations.  Ordering:
//   copy stream:  [job k-2 done] [job k-1 set up] upload Psi_k -> up[k % 2]
//   plan stream:  s0_k, m = v = 0 -> set up; [up[k % 2]] iterations; read back -> done[k % 2]
// The copy engine therefore takes a job's small initial-map copy before the
// next job's channel data, and a buffer is refilled only after the job that
// read it has finished.
#include "af_internal.cuh"

struct AfJobs {
    size_t iq_bytes = 0;
    void *iq[2] = {nullptr, nullptr};
    float *scale[2] = {nullptr, nullptr};
    float *s = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t up[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr}, setup = nullptr;
    long long count = 0;
};

void jobs_release(af_plan_t pl)
{
    AfJobs *j = pl->jobs;
    if (!j) return;
    if (j->copy) cudaStreamSynchronize(j->copy);
    for (int b = 0; b < 2; ++b) {
        if (j->iq[b]) cudaFree(j->iq[b]);
        if (j->scale[b]) cudaFree(j->scale[b]);
        if (j->up[b]) cudaEventDestroy(j->up[b]);
        if (j->done[b]) cudaEventDestroy(j->done[b]);
    }
    for (float *p : {j->s, j->grad, j->m, j->v, j->loss})
        if (p) cudaFree(p);
    if (j->setup) cudaEventDestroy(j->setup);
    if (j->copy) cudaStreamDestroy(j->copy);
    delete j;
    pl->jobs = nullptr;
}

extern "C" af_status af_job_reserve(af_plan_t pl)
{
    if (!pl) return af_set_error(AF_ERR_ARG, "af_job_reserve: plan is NULL");
    if (pl->jobs) return af_set_error(AF_OK, "");
    AfJobs *j = new AfJobs;
    pl->jobs = j;
    const size_t ne = pl->cfg.n_elem, ns = pl->cfg.n_samp, ng = (size_t)pl->g.ng;
    j->iq_bytes = ne * ne * ns * (pl->iq_dtype == AF_IQ_C64 ? 8 : 4);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc(&j->iq[b], j->iq_bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&j->scale[b], ne * sizeof(float));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->up[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done[b], cudaEventDisableTiming);
    }
    for (float **p : {&j->s, &j->grad, &j->m, &j->v})
        if (e == cudaSuccess) e = cudaMalloc((void **)p, ng * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&j->loss, 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->setup, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&j->copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        jobs_release(pl);
        return af_set_error(AF_ERR_CUDA, "af_job_reserve: %s", cudaGetErrorString(e));
    }
    return af_set_error(AF_OK, "");
}

extern "C" af_status af_job_submit(af_plan_t pl, const void *h_iq, const float *h_iq_scale, const float *h_s0,
                                   int n_iter, float *h_s_out, float *h_loss_out)
{
    if (!pl || !h_iq || !h_s0) return af_set_error(AF_ERR_ARG, "af_job_submit: NULL argument");
    if (n_iter < 1) return af_set_error(AF_ERR_ARG, "af_job_submit: n_iter = %d < 1", n_iter);
    const bool half = pl->iq_dtype != AF_IQ_C64;
    if (half && !h_iq_scale) return af_set_error(AF_ERR_DTYPE, "16-bit channel data needs h_iq_scale");
    if (!pl->jobs) {
        const af_status st = af_job_reserve(pl);
        if (st != AF_OK) return st;
    }
    AfJobs *j = pl->jobs;
    const size_t ng = (size_t)pl->g.ng, ne = pl->cfg.n_elem;
    const int b = (int)(j->count & 1);
    cudaStream_t st = pl->stream;
#define JOB_CUDA(call)                                                                                        \
    do {                                                                                                      \
        const cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_job_submit: %s", cudaGetErrorString(e_)); \
    } while (0)
    // upload of this job's channel data
    if (j->count >= 2) JOB_CUDA(cudaStreamWaitEvent(j->copy, j->done[b], 0));
    if (j->count >= 1) JOB_CUDA(cudaStreamWaitEvent(j->copy, j->setup, 0));
    JOB_CUDA(cudaMemcpyAsync(j->iq[b], h_iq, j->iq_bytes, cudaMemcpyHostToDevice, j->copy));
    if (half) JOB_CUDA(cudaMemcpyAsync(j->scale[b], h_iq_scale, ne * sizeof(float), cudaMemcpyHostToDevice, j->copy));
    JOB_CUDA(cudaEventRecord(j->up[b], j->copy));
    // initial state, then the iterations once the channel data is in
    JOB_CUDA(cudaMemcpyAsync(j->s, h_s0, ng * sizeof(float), cudaMemcpyHostToDevice, st));
    JOB_CUDA(cudaMemsetAsync(j->m, 0, ng * sizeof(float), st));
    JOB_CUDA(cudaMemsetAsync(j->v, 0, ng * sizeof(float), st));
    JOB_CUDA(cudaEventRecord(j->setup, st));
    JOB_CUDA(cudaStreamWaitEvent(st, j->up[b], 0));
    ++j->count;
    for (int it = 1; it <= n_iter; ++it) {
        const af_status s = af_iterate(pl, j->iq[b], half ? j->scale[b] : nullptr, j->s, j->grad, j->m, j->v, it,
                                       j->loss);
        if (s != AF_OK) {
            // whatever this job enqueued still reads buffer b: a later upload into it
            // must wait for that work too
            cudaEventRecord(j->done[b], st);
            return s;
        }
    }
    if (h_s_out) JOB_CUDA(cudaMemcpyAsync(h_s_out, j->s, ng * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (h_loss_out) JOB_CUDA(cudaMemcpyAsync(h_loss_out, j->loss, 4 * sizeof(float), cudaMemcpyDeviceToHost, st));
    JOB_CUDA(cudaEventRecord(j->done[b], st));
#undef JOB_CUDA
    return af_set_error(AF_OK, "");
}

extern "C" af_status af_job_wait(af_plan_t pl)
{
    if (!pl) return af_set_error(AF_ERR_ARG, "af_job_wait: plan is NULL");
    cudaError_t e = cudaSuccess;
    if (pl->jobs && pl->jobs->copy) e = cudaStreamSynchronize(pl->jobs->copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_job_wait: %s", cudaGetErrorString(e));
    return af_sync_status(pl);
}
