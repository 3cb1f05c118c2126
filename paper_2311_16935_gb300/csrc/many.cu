// osmodi_solve_many: a batch of independent problems, each solved by the
// full single-problem path (osmodi_solve: any scheme, precision and
// preconditioner of its plan), spread over several CUDA streams that as many
// host threads drive concurrently.  It complements osmodi_solve_batched (one
// persistent launch of plain CG over the whole batch): with the multigrid
// preconditioner each problem needs a few dozen iterations instead of
// thousands, and the streams keep the GPU busy while one problem's host
// thread waits for its convergence checks.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

extern "C" osmodi_status osmodi_solve_many(int count, const osmodi_plan* plans, const void* const* grads, int grad_dtype,
                                           void* const* ps, int p_dtype, double tol, int max_iter, int streams,
                                           void* const* workspaces, osmodi_result* results) {
    if (results && count > 0) std::memset(results, 0, sizeof(osmodi_result) * (size_t)count);
    if (count <= 0 || !plans || !grads || !ps || !workspaces || streams < 1 || streams > 64) return OSMODI_E_INVALID;
    int dev = -1;
    OSM_CUDA(cudaGetDevice(&dev));
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !grads[i] || !ps[i]) return OSMODI_E_INVALID;
        if (plans[i]->device != dev) return OSMODI_E_INVALID;
    }
    const int K = streams < count ? streams : count;
    // a plan holds per-solve host state (its mirror, graphs, events): one
    // plan listed twice must land on the same stream, whose thread solves
    // its problems one after the other
    {
        std::unordered_map<osmodi_plan, int> stream_of;
        for (int i = 0; i < count; ++i) {
            auto it = stream_of.emplace(plans[i], i % K).first;
            if (it->second != i % K) return OSMODI_E_INVALID;
        }
    }
    for (int w = 0; w < K; ++w) {
        if (!workspaces[w]) return OSMODI_E_WORKSPACE;
        // the caller sizes workspaces[w] for every problem of stream w (this
        // interface takes no sizes, so a short one cannot be detected here);
        // only plans that report no workspace size are refused
        for (int i = w; i < count; i += K)
            if (osmodi_workspace_bytes(plans[i]) == 0) return OSMODI_E_INVALID;
    }
    std::vector<osmodi_status> st(count, OSMODI_OK);
    std::vector<std::string> err(K);
    std::atomic<int> failed{0};
    auto worker = [&](int w) {
        if (cudaSetDevice(dev) != cudaSuccess) {
            err[w] = "cudaSetDevice in a solve_many worker";
            failed.store(1);
            return;
        }
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            err[w] = "cudaStreamCreateWithFlags in a solve_many worker";
            failed.store(1);
            return;
        }
        // problem i always goes to stream i mod K, so a plan's captured CUDA
        // graphs always see the same workspace
        for (int i = w; i < count; i += K) {
            if (failed.load()) break;
            osmodi_result* r = results ? &results[i] : nullptr;
            st[i] = osmodi_solve(plans[i], grads[i], grad_dtype, ps[i], p_dtype, tol, max_iter, workspaces[w], s, r);
            if (st[i] < 0 && st[i] != OSMODI_E_NAN_INPUT) {
                err[w] = osm::last_cuda_error();
                failed.store(1);
            }
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    pool.reserve(K);
    for (int w = 0; w < K; ++w) pool.emplace_back(worker, w);
    for (auto& t : pool) t.join();
    osmodi_status overall = OSMODI_OK;
    for (int i = 0; i < count; ++i) {
        if (st[i] < 0 && st[i] != OSMODI_E_NAN_INPUT) {
            overall = st[i];
            break;
        }
        if (st[i] == OSMODI_E_NAN_INPUT && overall >= 0) overall = st[i];
        else if (st[i] == OSMODI_NOT_CONVERGED && overall == OSMODI_OK) overall = st[i];
    }
    for (int w = 0; w < K; ++w)
        if (!err[w].empty()) {
            osm::set_error_text(err[w].c_str());
            break;
        }
    return overall;
}
