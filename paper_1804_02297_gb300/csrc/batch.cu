// Batches of independent problems of uneven size (different n, k and media).
//
// Each problem keeps its own stream, workspaces, stencils and factor.  The
// batched apply forks one branch per problem from the caller's stream and joins
// them back; after a first direct run (which also sizes every workspace) the
// fork/join is captured once into a CUDA graph and replayed by later calls with
// the same buffers, so a batch of many small problems costs one graph launch.
// Batched set-up and solves run concurrently from a pool of host threads, each
// problem on its own stream.
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"

struct spm_batch_s {
    std::vector<spm_problem_s *> probs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaEvent_t fork = nullptr;
    // cached graph of the batched apply
    int g_prec = -1;
    std::vector<const void *> g_x;
    std::vector<void *> g_y;
    cudaGraphExec_t g_exec = nullptr;
};

namespace {

template <typename F> spm_status parallel_for(int count, F fn)
{
    int nthreads = (int)std::thread::hardware_concurrency();
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 8) nthreads = 8;
    if (nthreads > count) nthreads = count;
    std::atomic<int> next(0);
    std::atomic<int> first_err(SPM_OK);
    std::vector<std::thread> pool;
    char msg[1024] = "";
    std::atomic<int> msg_set(0);
    for (int w = 0; w < nthreads; ++w)
        pool.emplace_back([&]() {
            for (;;) {
                int i = next.fetch_add(1);
                if (i >= count) break;
                spm_status st = fn(i);
                if (st != SPM_OK) {
                    int expected = SPM_OK;
                    if (first_err.compare_exchange_strong(expected, (int)st) && !msg_set.exchange(1))
                        snprintf(msg, sizeof(msg), "problem %d: %s", i, spm_last_error());
                }
            }
        });
    for (auto &t : pool) t.join();
    if (first_err.load() != SPM_OK) spm_set_error("%s", msg);
    return (spm_status)first_err.load();
}

spm_status fork_join_apply(spm_batch_s *B, int prec, const void *const *x, void *const *y, cudaStream_t s)
{
    SPM_CUDA_TRY(cudaEventRecord(B->fork, s));
    for (size_t i = 0; i < B->probs.size(); ++i) {
        SPM_CUDA_TRY(cudaStreamWaitEvent(B->streams[i], B->fork, 0));
        SPM_TRY(spm_apply_A_impl(B->probs[i], prec, x[i], y[i], 1, B->streams[i]));
        SPM_CUDA_TRY(cudaEventRecord(B->events[i], B->streams[i]));
        SPM_CUDA_TRY(cudaStreamWaitEvent(s, B->events[i], 0));
    }
    return SPM_OK;
}

} // namespace

extern "C" spm_status spm_destroy_batch(spm_batch B)
{
    if (!B) return SPM_OK;
    if (B->g_exec) cudaGraphExecDestroy(B->g_exec);
    for (auto *P : B->probs) spm_destroy(P);
    for (auto s : B->streams) if (s) cudaStreamDestroy(s);
    for (auto e : B->events) if (e) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    delete B;
    return SPM_OK;
}

extern "C" spm_status spm_create_batch(int count, const int *n, const double *omega, const double *const *eps_host,
                                       const double *const *grad_eps_host, spm_quad quad, spm_batch *out)
{
    if (!out || count <= 0 || !n || !omega || !eps_host) { spm_set_error("bad batch arguments"); return SPM_ERR_INVALID_ARG; }
    *out = nullptr;
    spm_batch_s *B = new spm_batch_s();
    B->probs.assign(count, nullptr);
    B->streams.assign(count, nullptr);
    B->events.assign(count, nullptr);
    auto fail = [&](spm_status st) { spm_destroy_batch(B); return st; };
    if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) { spm_set_error("event create failed"); return fail(SPM_ERR_CUDA); }
    for (int i = 0; i < count; ++i) {
        if (cudaStreamCreateWithFlags(&B->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->events[i], cudaEventDisableTiming) != cudaSuccess) {
            spm_set_error("stream/event create failed");
            return fail(SPM_ERR_CUDA);
        }
    }
    spm_status st = parallel_for(count, [&](int i) {
        return spm_create_problem(n[i], omega[i], eps_host[i], grad_eps_host ? grad_eps_host[i] : nullptr, quad,
                                  B->streams[i], &B->probs[i]);
    });
    if (st != SPM_OK) return fail(st);
    *out = B;
    return SPM_OK;
}

extern "C" spm_status spm_batch_size(spm_batch B, int *count)
{
    if (!B || !count) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    *count = (int)B->probs.size();
    return SPM_OK;
}

extern "C" spm_status spm_batch_problem(spm_batch B, int index, spm_problem *out)
{
    if (!B || !out || index < 0 || index >= (int)B->probs.size()) { spm_set_error("bad batch index"); return SPM_ERR_INVALID_ARG; }
    *out = B->probs[index];
    return SPM_OK;
}

extern "C" spm_status spm_batch_build_stencils(spm_batch B, spm_prec factor_prec)
{
    if (!B) { spm_set_error("NULL batch"); return SPM_ERR_INVALID_ARG; }
    // Up to 8 problems are factored at once, each with its own front and update
    // workspaces; a problem whose workspace did not fit beside the others is
    // factored again afterwards, alone.
    const int count = (int)B->probs.size();
    std::vector<int> status(count, SPM_OK);
    parallel_for(count, [&](int i) -> spm_status {
        status[i] = spm_build_stencils(B->probs[i], factor_prec);
        return status[i] == SPM_ERR_OOM ? SPM_OK : (spm_status)status[i];
    });
    for (int i = 0; i < count; ++i)
        if (status[i] != SPM_OK && status[i] != SPM_ERR_OOM) {
            spm_set_error("problem %d: build failed (status %d)", i, status[i]);
            return (spm_status)status[i];
        }
    for (int i = 0; i < count; ++i)
        if (status[i] == SPM_ERR_OOM) {
            cudaDeviceSynchronize();
            spm_status st = spm_build_stencils(B->probs[i], factor_prec);
            if (st != SPM_OK) {
                char msg[1024];
                snprintf(msg, sizeof(msg), "problem %d: %s", i, spm_last_error());
                spm_set_error("%s", msg);
                return st;
            }
        }
    return SPM_OK;
}

extern "C" spm_status spm_batch_apply_A(spm_batch B, spm_prec prec, const void *const *x_dev, void *const *y_dev,
                                        void *stream)
{
    if (!B || !x_dev || !y_dev) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    if (prec != SPM_C128 && prec != SPM_C64) { spm_set_error("apply precision must be SPM_C128 or SPM_C64"); return SPM_ERR_INVALID_ARG; }
    const size_t cnt = B->probs.size();
    for (size_t i = 0; i < cnt; ++i)
        if (!x_dev[i] || !y_dev[i] || x_dev[i] == y_dev[i]) { spm_set_error("bad buffer for problem %zu", i); return SPM_ERR_INVALID_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    bool same = B->g_exec && B->g_prec == (int)prec && B->g_x.size() == cnt;
    for (size_t i = 0; same && i < cnt; ++i) same = B->g_x[i] == x_dev[i] && B->g_y[i] == y_dev[i];
    if (same) {
        SPM_CUDA_TRY(cudaGraphLaunch(B->g_exec, s));
        return SPM_OK;
    }
    // direct run (sizes every workspace), then capture the same fork/join for replay
    SPM_TRY(fork_join_apply(B, prec, x_dev, y_dev, s));
    if (B->g_exec) { cudaGraphExecDestroy(B->g_exec); B->g_exec = nullptr; }
    cudaStream_t cap;
    SPM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    spm_status st = SPM_OK;
    if (e == cudaSuccess) {
        st = fork_join_apply(B, prec, x_dev, y_dev, cap);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess && st == SPM_OK) e = cudaGraphInstantiate(&B->g_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (st != SPM_OK) return st;
    if (e != cudaSuccess) {
        B->g_exec = nullptr;
        spm_set_error("capturing the batched apply failed: %s", cudaGetErrorString(e));
        return SPM_ERR_CUDA;
    }
    B->g_prec = (int)prec;
    B->g_x.assign(x_dev, x_dev + cnt);
    B->g_y.assign(y_dev, y_dev + cnt);
    return SPM_OK;
}

extern "C" spm_status spm_batch_solve(spm_batch B, spm_prec prec, const void *const *g_dev, void *const *x_dev,
                                      double tol, int maxit, int restart, spm_solve_info *infos)
{
    if (!B || !g_dev || !x_dev) { spm_set_error("NULL argument"); return SPM_ERR_INVALID_ARG; }
    return parallel_for((int)B->probs.size(), [&](int i) {
        return spm_solve(B->probs[i], prec, g_dev[i], x_dev[i], 1, tol, maxit, restart, infos ? &infos[i] : nullptr);
    });
}
