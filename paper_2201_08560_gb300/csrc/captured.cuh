// Host-side helpers of the level-synchronous drivers: a pinned flag read and
// the captured round loop (a CUDA graph of several gated rounds, replayed
// until a device flag reads 0).
#pragma once

#include "b2sr_internal.cuh"

namespace b2sr {

// Pinned host word for loop-exit flags.
struct HostFlag {
    int32_t* p = nullptr;
    HostFlag() { if (cudaMallocHost(&p, sizeof(int32_t)) != cudaSuccess) { cudaGetLastError(); p = nullptr; } }
    ~HostFlag() { if (p) cudaFreeHost(p); }
};

inline b2sr_status read_flag(const int32_t* dev, HostFlag& hf, cudaStream_t s, int32_t* out) {
    if (!hf.p) return fail(B2SR_ERR_OOM, "pinned flag");
    B2SR_CUDA_TRY(cudaMemcpyAsync(hf.p, dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    B2SR_CUDA_TRY(cudaStreamSynchronize(s));
    *out = *hf.p;
    return B2SR_OK;
}

__device__ __forceinline__ bool gate_closed(const int32_t* gate) { return gate && *gate == 0; }

// ---------------------------------------------------------------------------
// captured round loop
// ---------------------------------------------------------------------------
// Enqueues `per_graph` rounds (body(stream, r)) into one CUDA graph on a
// private stream, then replays it until *active reads 0.  Every round must be
// gated on *active.  Returns in *rounds the rounds replayed; B2SR_ERR_NOT_CONVERGED
// if *active is still set after max_rounds.
template <class Body>
b2sr_status run_captured(cudaStream_t user, int per_graph, int64_t max_rounds, const int32_t* active,
                                Body&& body, int64_t* rounds) {
    *rounds = 0;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    HostFlag hf;
    auto cleanup = [&](b2sr_status st) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) {
            if (ev) {  // the caller's stream waits for everything enqueued here
                cudaEventRecord(ev, cs);
                cudaStreamWaitEvent(user, ev, 0);
            }
            cudaStreamDestroy(cs);
        }
        if (ev) cudaEventDestroy(ev);
        return st;
    };
    B2SR_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaEventCreate"));
    e = cudaEventRecord(ev, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "order capture stream"));
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamBeginCapture"));
    const int64_t l0 = b2sr_launch_count();
    b2sr_status st = B2SR_OK;
    for (int r = 0; r < per_graph && st == B2SR_OK; ++r) st = body(cs, r);
    e = cudaStreamEndCapture(cs, &graph);
    if (st != B2SR_OK) return cleanup(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamEndCapture"));
    const int64_t per_replay = b2sr_launch_count() - l0;
    note_launches(-per_replay);  // counted again per replay below
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaGraphInstantiate"));
    for (;;) {
        e = cudaGraphLaunch(exec, cs);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaGraphLaunch"));
        note_launches(per_replay);
        *rounds += per_graph;
        int32_t got = 0;
        st = read_flag(active, hf, cs, &got);
        if (st != B2SR_OK) return cleanup(st);
        if (!got) return cleanup(B2SR_OK);
        if (*rounds >= max_rounds) return cleanup(fail(B2SR_ERR_NOT_CONVERGED, "exceeded max_iters rounds"));
    }
}

}  // namespace b2sr
