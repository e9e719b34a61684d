// Query serving over resident B2SR graphs: BFS and PageRank queries (Sec. V
// drivers) batched continuously on the device.
//
//   * Registry: graphs are added once and stay resident; their bytes count
//     against the server's device-memory budget.
//   * Admission: a query waits in its graph's queue until a batch slot is
//     free and the batch's working memory fits the budget; a query whose
//     batch could never fit is refused at submission.
//   * BFS queries on one graph share a 64-lane batch: lane s of the uint64
//     frontier, visited and next words (b2sr_spmm_bits64) is one query.  New
//     queries take free lanes at the next level boundary; a lane retires when
//     its level finds no new vertex.  Each lane has its own depth, so queries
//     that joined at different times advance together.
//   * PageRank queries on one graph share blocks of four fp32 columns
//     (b2sr_spmm_f32x4); a column joins at the next iteration boundary and
//     retires after its own iteration count.  A query is the uniform-teleport
//     PageRank (source < 0) or the personalised one with all teleport mass on
//     its source.
//   * One worker thread drives all graphs, each on its own stream: it issues a
//     step (one BFS level and one PageRank iteration for every active slot),
//     then moves on to the next graph, and collects a graph's step when its
//     event has completed, so steps of different graphs overlap on the device.
// Every per-lane and per-column computation is independent of the others in
// its batch and uses a fixed reduction order, so a query's result is the same
// alone and in any mix: bit-exact levels, and PageRank bitwise equal to
// b2sr_pagerank with the same teleport vector.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "b2sr_internal.cuh"

namespace b2sr {
b2sr_status spmm64_dispatch(b2sr_matrix* h, const uint64_t* X, uint64_t* Y, const uint64_t* M, int comp,
                            cudaStream_t s, const int32_t* gate);
b2sr_status spmm4_dispatch(b2sr_matrix* h, const float* X, float* Y, const uint32_t* M, int comp, cudaStream_t s,
                           const int32_t* gate);

using Clock = std::chrono::steady_clock;

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
struct LaneArgs {
    int32_t* out[64];   // levels output of each lane's query
    int32_t src[64];
    int32_t depth[64];  // level of the lane's current frontier
};

// New lanes: clear their bits, seed their sources, fill their outputs.
__global__ void lane_init_kernel(unsigned long long* X, unsigned long long* V, int32_t n, unsigned long long fresh,
                                 LaneArgs a) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long x = X[v] & ~fresh, vis = V[v] & ~fresh;
        unsigned long long b = fresh;
        while (b) {
            const int s = __ffsll((long long)b) - 1;
            b &= b - 1;
            const bool is_src = a.src[s] == v;
            a.out[s][v] = is_src ? 0 : -1;
            if (is_src) {
                x |= 1ull << s;
                vis |= 1ull << s;
            }
        }
        X[v] = x;
        V[v] = vis;
    }
}

// visited |= next; new vertices of lane s get level depth[s] + 1; found = OR of next
__global__ void lane_update_kernel(const unsigned long long* __restrict__ Y, unsigned long long* __restrict__ V,
                                   int32_t n, LaneArgs a, unsigned long long* found) {
    unsigned long long any = 0ull;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long b = Y[v];
        if (!b) continue;
        any |= b;
        V[v] |= b;
        while (b) {
            const int s = __ffsll((long long)b) - 1;
            b &= b - 1;
            a.out[s][v] = a.depth[s] + 1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) any |= __shfl_xor_sync(0xffffffffu, any, o);
    if ((threadIdx.x & 31) == 0 && any) atomicOr(found, any);
}

struct ColArgs {
    int32_t src[4];   // < 0: uniform teleport
    float damp[4];
    float* out[4];    // written when the column finishes in this step
    uint32_t init;    // columns starting in this step
    uint32_t step;    // columns taking an iteration in this step
    uint32_t finish;  // columns whose result is copied out after this step
};

// x^0 = 1/n and c = x / outdeg for the starting columns (the arithmetic of b2sr_pagerank)
__global__ void col_init_kernel(float* Pr, float* C, const int32_t* __restrict__ outdeg, int32_t n, ColArgs a) {
    const float x0 = __fdiv_rn(1.0f, (float)n);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = outdeg[v];
        const float c0 = d > 0 ? __fdiv_rn(x0, (float)d) : 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (a.init >> b & 1u) {
                Pr[4 * v + b] = x0;
                C[4 * v + b] = c0;
            }
    }
}

// x = (1-d) t + d y; c = x / outdeg; finished columns copied out
__global__ void col_step_kernel(const float* __restrict__ Y, float* Pr, float* C, const int32_t* __restrict__ outdeg,
                                int32_t n, ColArgs a) {
    const float tu = __fdiv_rn(1.0f, (float)n);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = outdeg[v];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (a.step >> b & 1u) {
                const float t = a.src[b] < 0 ? tu : (a.src[b] == v ? 1.0f : 0.0f);
                const float x = __fmaf_rn(a.damp[b], Y[4 * v + b], __fmul_rn(1.0f - a.damp[b], t));
                Pr[4 * v + b] = x;
                C[4 * v + b] = d > 0 ? __fdiv_rn(x, (float)d) : 0.0f;
            }
            if (a.finish >> b & 1u) a.out[b][v] = Pr[4 * v + b];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
enum QState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3 };

struct QueryRec {
    int64_t id = 0;
    int kind = 0;  // 0 BFS, 1 PageRank
    int graph = 0;
    int32_t src = 0;
    int iters = 0;
    float damp = 0.85f;
    void* out = nullptr;
    Clock::time_point t_submit, t_done;
    std::atomic<int> state{Q_QUEUED};
    b2sr_status status = B2SR_OK;
};

struct PRBlock {
    float* Pr = nullptr;
    float* C = nullptr;
    float* Y = nullptr;
    QueryRec* col[4] = {nullptr, nullptr, nullptr, nullptr};
    int done_it[4] = {0, 0, 0, 0};  // iterations issued
    bool fresh[4] = {false, false, false, false};
    uint32_t finishing = 0;         // columns that complete with the step in flight
};

struct GraphSlot {
    b2sr_matrix* h = nullptr;
    int64_t bytes = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    unsigned long long* found_host = nullptr;  // pinned
    bool in_flight = false;
    std::deque<QueryRec*> pend_bfs, pend_pr;
    // BFS batch
    void* bfs_mem = nullptr;  // the allocation holding X, Y, V, found (X and Y swap every level)
    unsigned long long *X = nullptr, *Y = nullptr, *V = nullptr, *found = nullptr;
    int64_t bfs_bytes = 0;
    QueryRec* lane[64] = {};
    int32_t depth[64] = {};
    unsigned long long active = 0ull, fresh = 0ull;
    bool bfs_stepped = false;
    // PageRank blocks
    std::vector<PRBlock> blocks;
    int64_t block_bytes = 0;
};

}  // namespace b2sr

struct b2sr_server {
    int device = 0;
    int64_t budget = 0;
    int64_t used = 0;  // resident graphs + batch state
    int max_lanes = 64;
    int max_blocks = 2;
    std::vector<std::unique_ptr<b2sr::GraphSlot>> graphs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<b2sr::QueryRec*> inbox;
    std::unordered_map<int64_t, std::unique_ptr<b2sr::QueryRec>> queries;
    int64_t next_id = 1;
    std::thread worker;
    bool stop = false;
    int64_t outstanding = 0;  // submitted and not yet finished
    // statistics since the last reset
    std::vector<double> lat_us;
    int64_t submitted = 0, completed = 0, failed = 0, refused = 0, steps = 0;
    b2sr::Clock::time_point t0, t_last;
    bool have_t0 = false;
    std::string worker_error;
};

namespace b2sr {

static int64_t partial_bytes(const b2sr_matrix* h, int value_bytes) {
    return 2 * (h->nchunks + 1) * (int64_t)h->k * value_bytes + 4096;
}
static int64_t bfs_state_bytes(const b2sr_matrix* h) {
    return 3 * (int64_t)h->n * 8 + 256 + partial_bytes(h, 8);
}
static int64_t block_state_bytes(const b2sr_matrix* h) {
    return 3 * (int64_t)h->n * 16 + 3 * 256 + partial_bytes(h, 16);
}

static void finish(b2sr_server* S, QueryRec* q, b2sr_status st) {
    q->t_done = Clock::now();
    q->status = st;
    q->state.store(st == B2SR_OK ? Q_DONE : Q_FAILED);
    std::lock_guard<std::mutex> lk(S->mu);
    S->outstanding--;
    if (st == B2SR_OK) {
        S->completed++;
        S->lat_us.push_back(std::chrono::duration<double, std::micro>(q->t_done - q->t_submit).count());
        S->t_last = q->t_done;
    } else {
        S->failed++;
    }
    S->cv_done.notify_all();
}

// Fails every query the graph holds (after a CUDA error on its stream).
static void fail_graph(b2sr_server* S, GraphSlot& g, b2sr_status st) {
    for (int s = 0; s < 64; ++s)
        if (g.lane[s]) { finish(S, g.lane[s], st); g.lane[s] = nullptr; }
    g.active = g.fresh = 0ull;
    for (auto& b : g.blocks)
        for (int c = 0; c < 4; ++c)
            if (b.col[c]) { finish(S, b.col[c], st); b.col[c] = nullptr; }
    for (auto* q : g.pend_bfs) finish(S, q, st);
    for (auto* q : g.pend_pr) finish(S, q, st);
    g.pend_bfs.clear();
    g.pend_pr.clear();
}

static bool reserve(b2sr_server* S, int64_t bytes) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->used + bytes > S->budget) return false;
    S->used += bytes;
    return true;
}
static void release(b2sr_server* S, int64_t bytes) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= bytes;
}

// Pending queries take free lanes and columns (allocating batch state under the budget).
static b2sr_status admit(b2sr_server* S, GraphSlot& g) {
    const int32_t n = g.h->n;
    while (!g.pend_bfs.empty()) {
        if (!g.X) {
            if (!reserve(S, g.bfs_bytes)) break;
            DevBuf tmp(g.st);
            b2sr_status st = tmp.alloc(3 * (size_t)n * 8 + 256);
            if (st != B2SR_OK) { release(S, g.bfs_bytes); return st; }
            g.bfs_mem = tmp.p;
            g.X = tmp.as<unsigned long long>();
            g.Y = g.X + n;
            g.V = g.Y + n;
            g.found = g.V + n;
            tmp.p = nullptr;  // owned by the slot now
            B2SR_CUDA_TRY(cudaMemsetAsync(g.X, 0, 3 * (size_t)n * 8 + 8, g.st));
        }
        const unsigned long long busy = g.active | g.fresh;
        if (__builtin_popcountll(busy) >= S->max_lanes) break;
        const int s = __builtin_ctzll(~busy);
        QueryRec* q = g.pend_bfs.front();
        g.pend_bfs.pop_front();
        q->state.store(Q_RUNNING);
        g.lane[s] = q;
        g.depth[s] = 0;
        g.fresh |= 1ull << s;
    }
    while (!g.pend_pr.empty()) {
        PRBlock* blk = nullptr;
        int col = -1;
        for (auto& b : g.blocks) {
            for (int c = 0; c < 4 && col < 0; ++c)
                if (!b.col[c]) col = c;
            if (col >= 0) { blk = &b; break; }
        }
        if (!blk) {
            if ((int)g.blocks.size() >= S->max_blocks || !reserve(S, g.block_bytes)) break;
            DevBuf tmp(g.st);
            const size_t vb = round_up((size_t)n * 16, 256);
            b2sr_status st = tmp.alloc(3 * vb);
            if (st != B2SR_OK) { release(S, g.block_bytes); return st; }
            PRBlock b;
            b.Pr = tmp.as<float>();
            b.C = reinterpret_cast<float*>(tmp.as<char>() + vb);
            b.Y = reinterpret_cast<float*>(tmp.as<char>() + 2 * vb);
            tmp.p = nullptr;
            B2SR_CUDA_TRY(cudaMemsetAsync(b.Pr, 0, 3 * vb, g.st));
            g.blocks.push_back(b);
            blk = &g.blocks.back();
            col = 0;
        }
        QueryRec* q = g.pend_pr.front();
        g.pend_pr.pop_front();
        q->state.store(Q_RUNNING);
        blk->col[col] = q;
        blk->done_it[col] = 0;
        blk->fresh[col] = true;
    }
    return B2SR_OK;
}

// Frees batch state a graph no longer uses.
static void trim(b2sr_server* S, GraphSlot& g) {
    if (g.X && !g.active && !g.fresh && g.pend_bfs.empty()) {
        dfree(g.bfs_mem, g.st);
        g.bfs_mem = nullptr;
        g.X = g.Y = g.V = g.found = nullptr;
        release(S, g.bfs_bytes);
    }
    for (size_t i = g.blocks.size(); i-- > 0;) {
        PRBlock& b = g.blocks[i];
        if (!b.col[0] && !b.col[1] && !b.col[2] && !b.col[3] && g.pend_pr.empty()) {
            dfree(b.Pr, g.st);
            g.blocks.erase(g.blocks.begin() + i);
            release(S, g.block_bytes);
        }
    }
}

// Enqueues one step on the graph's stream: a BFS level for the active and
// new lanes, a PageRank iteration for every busy column.
static b2sr_status launch_step(GraphSlot& g) {
    const int32_t n = g.h->n;
    g.bfs_stepped = false;
    if (g.active | g.fresh) {
        LaneArgs la;
        for (int s = 0; s < 64; ++s) {
            la.out[s] = g.lane[s] ? static_cast<int32_t*>(g.lane[s]->out) : nullptr;
            la.src[s] = g.lane[s] ? g.lane[s]->src : -1;
            la.depth[s] = g.depth[s];
        }
        if (g.fresh) {
            lane_init_kernel<<<grid_for(n), 256, 0, g.st>>>(g.X, g.V, n, g.fresh, la);
            B2SR_LAUNCH_CHECK("lane_init_kernel");
            g.active |= g.fresh;
            g.fresh = 0ull;
        }
        B2SR_TRY(spmm64_dispatch(g.h, reinterpret_cast<uint64_t*>(g.X), reinterpret_cast<uint64_t*>(g.Y),
                                 reinterpret_cast<uint64_t*>(g.V), 1, g.st, nullptr));
        B2SR_CUDA_TRY(cudaMemsetAsync(g.found, 0, 8, g.st));
        lane_update_kernel<<<grid_for(n), 256, 0, g.st>>>(g.Y, g.V, n, la, g.found);
        B2SR_LAUNCH_CHECK("lane_update_kernel");
        std::swap(g.X, g.Y);
        B2SR_CUDA_TRY(cudaMemcpyAsync(g.found_host, g.found, 8, cudaMemcpyDeviceToHost, g.st));
        g.bfs_stepped = true;
    }
    for (auto& b : g.blocks) {
        ColArgs ca{};
        for (int c = 0; c < 4; ++c) {
            QueryRec* q = b.col[c];
            ca.src[c] = q ? q->src : -1;
            ca.damp[c] = q ? q->damp : 0.0f;
            ca.out[c] = q ? static_cast<float*>(q->out) : nullptr;
            if (!q) continue;
            if (b.fresh[c]) ca.init |= 1u << c;
            if (b.done_it[c] < q->iters) ca.step |= 1u << c;
            if (b.done_it[c] + 1 >= q->iters) ca.finish |= 1u << c;  // iters == 0: copied right after init
        }
        if (!(ca.init | ca.step | ca.finish)) continue;
        if (ca.init) {
            col_init_kernel<<<grid_for(n), 256, 0, g.st>>>(b.Pr, b.C, g.h->outdeg, n, ca);
            B2SR_LAUNCH_CHECK("col_init_kernel");
        }
        if (ca.step) B2SR_TRY(spmm4_dispatch(g.h, b.C, b.Y, nullptr, 0, g.st, nullptr));
        col_step_kernel<<<grid_for(n), 256, 0, g.st>>>(b.Y, b.Pr, b.C, g.h->outdeg, n, ca);
        B2SR_LAUNCH_CHECK("col_step_kernel");
        for (int c = 0; c < 4; ++c) {
            b.fresh[c] = false;
            if (ca.step >> c & 1u) b.done_it[c]++;
        }
        b.finishing = ca.finish;
    }
    B2SR_CUDA_TRY(cudaEventRecord(g.ev, g.st));
    g.in_flight = true;
    return B2SR_OK;
}

// The step in flight has completed: retire lanes and columns that are done.
static void collect(b2sr_server* S, GraphSlot& g) {
    g.in_flight = false;
    if (g.bfs_stepped) {
        const unsigned long long f = *g.found_host;
        for (int s = 0; s < 64; ++s) {
            if (!(g.active >> s & 1ull)) continue;
            g.depth[s]++;
            if (!(f >> s & 1ull)) {
                finish(S, g.lane[s], B2SR_OK);
                g.lane[s] = nullptr;
                g.active &= ~(1ull << s);
            }
        }
    }
    for (auto& b : g.blocks) {
        for (int c = 0; c < 4; ++c)
            if (b.finishing >> c & 1u) {
                finish(S, b.col[c], B2SR_OK);
                b.col[c] = nullptr;
            }
        b.finishing = 0;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->steps++;
}

static bool has_work(const GraphSlot& g) {
    if (g.active || g.fresh) return true;
    for (const auto& b : g.blocks)
        for (int c = 0; c < 4; ++c)
            if (b.col[c]) return true;
    return false;
}

static void worker_main(b2sr_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            bool busy = false;
            for (auto& gp : S->graphs)
                if (gp->in_flight || has_work(*gp) || !gp->pend_bfs.empty() || !gp->pend_pr.empty()) busy = true;
            if (!busy && S->inbox.empty()) {
                S->cv_work.wait(lk, [&] { return S->stop || !S->inbox.empty(); });
                if (S->stop) break;
            }
            while (!S->inbox.empty()) {
                QueryRec* q = S->inbox.front();
                S->inbox.pop_front();
                GraphSlot& g = *S->graphs[q->graph];
                (q->kind == 0 ? g.pend_bfs : g.pend_pr).push_back(q);
            }
        }
        bool progressed = false;
        for (auto& gp : S->graphs) {
            GraphSlot& g = *gp;
            if (g.in_flight) {
                const cudaError_t e = cudaEventQuery(g.ev);
                if (e == cudaErrorNotReady) continue;
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    g.in_flight = false;
                    {
                        std::lock_guard<std::mutex> lk(S->mu);
                        S->worker_error = cudaGetErrorString(e);
                    }
                    fail_graph(S, g, B2SR_ERR_CUDA);
                    continue;
                }
                collect(S, g);
                progressed = true;
            }
            b2sr_status st = admit(S, g);
            if (st == B2SR_OK && has_work(g)) st = launch_step(g);
            if (st != B2SR_OK) {
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->worker_error = b2sr_last_error();
                }
                cudaStreamSynchronize(g.st);
                g.in_flight = false;
                fail_graph(S, g, st);
            } else if (g.in_flight) {
                progressed = true;
            }
            if (!g.in_flight) trim(S, g);
        }
        if (!progressed) std::this_thread::yield();  // steps in flight: poll their events
    }
    for (auto& gp : S->graphs) {
        GraphSlot& g = *gp;
        if (g.in_flight) cudaEventSynchronize(g.ev);
        fail_graph(S, g, B2SR_ERR_ABORTED);
        trim(S, g);
        cudaStreamSynchronize(g.st);
    }
}

static b2sr_status check_server(const b2sr_server* S) {
    return S ? B2SR_OK : fail(B2SR_ERR_INVALID_ARG, "server is NULL");
}

static b2sr_status enqueue(b2sr_server* S, QueryRec* rec, int64_t need, int64_t* id) {
    std::unique_ptr<QueryRec> q(rec);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(B2SR_ERR_ABORTED, "server is stopping");
    // refuse only what could never fit beside the resident graphs; the rest
    // waits until batch memory frees up
    int64_t resident = 0;
    for (auto& g : S->graphs) resident += g->bytes;
    if (need > S->budget - resident) {
        S->refused++;
        return fail(B2SR_ERR_ADMISSION_REFUSED, "query batch needs " + std::to_string(need) +
                                                    " bytes; the budget beside the resident graphs is " +
                                                    std::to_string(S->budget - resident));
    }
    q->id = S->next_id++;
    q->t_submit = Clock::now();
    if (!S->have_t0) { S->t0 = q->t_submit; S->have_t0 = true; }
    *id = q->id;
    S->submitted++;
    S->outstanding++;
    S->inbox.push_back(q.get());
    S->queries.emplace(q->id, std::move(q));
    S->cv_work.notify_one();
    return B2SR_OK;
}

}  // namespace b2sr

using namespace b2sr;

extern "C" b2sr_status b2sr_server_create(int64_t budget_bytes, int max_bfs_lanes, int max_pr_blocks,
                                          b2sr_server_t* out) {
    clear_error();
    if (!out) return fail(B2SR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (budget_bytes <= 0 || max_bfs_lanes < 1 || max_bfs_lanes > 64 || max_pr_blocks < 0)
        return fail(B2SR_ERR_INVALID_ARG, "need budget > 0, 1 <= lanes <= 64, blocks >= 0");
    auto* S = new (std::nothrow) b2sr_server();
    if (!S) return fail(B2SR_ERR_OOM, "server");
    B2SR_CUDA_TRY(cudaGetDevice(&S->device));
    S->budget = budget_bytes;
    S->max_lanes = max_bfs_lanes;
    S->max_blocks = max_pr_blocks;
    S->worker = std::thread(worker_main, S);
    *out = S;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_server_add_graph(b2sr_server_t S, b2sr_handle h, int32_t* graph_id) {
    clear_error();
    B2SR_TRY(check_server(S));
    B2SR_TRY(check_handle(h));
    if (!graph_id) return fail(B2SR_ERR_INVALID_ARG, "graph_id is NULL");
    if (h->device != S->device) return fail(B2SR_ERR_INVALID_ARG, "graph lives on another device");
    auto g = std::make_unique<GraphSlot>();
    g->h = h;
    B2SR_CUDA_TRY(cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking));
    auto cleanup = [&](b2sr_status st) {
        if (g->found_host) cudaFreeHost(g->found_host);
        if (g->ev) cudaEventDestroy(g->ev);
        if (g->st) cudaStreamDestroy(g->st);
        return st;
    };
    cudaError_t e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&g->found_host, sizeof(unsigned long long));
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "server graph slot"));
    b2sr_status st = ensure_outdeg(h, g->st);  // PageRank needs it; built once, part of the resident bytes
    if (st != B2SR_OK) return cleanup(st);
    g->bytes = 4 * ((int64_t)h->ntr + 1) + h->cap * (4 + tile_bytes(h->k)) + 4 * (int64_t)h->n;
    g->bfs_bytes = bfs_state_bytes(h);
    g->block_bytes = block_state_bytes(h);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->used + g->bytes > S->budget) {
        S->refused++;
        return cleanup(fail(B2SR_ERR_ADMISSION_REFUSED, "graph does not fit the server's memory budget"));
    }
    S->used += g->bytes;
    *graph_id = (int32_t)S->graphs.size();
    S->graphs.push_back(std::move(g));
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_server_graph_bytes(b2sr_server_t S, int32_t graph, int64_t* resident,
                                               int64_t* bfs_batch, int64_t* pr_block) {
    clear_error();
    B2SR_TRY(check_server(S));
    std::lock_guard<std::mutex> lk(S->mu);
    if (graph < 0 || graph >= (int32_t)S->graphs.size()) return fail(B2SR_ERR_INVALID_ARG, "no such graph");
    const GraphSlot& g = *S->graphs[graph];
    if (resident) *resident = g.bytes;
    if (bfs_batch) *bfs_batch = g.bfs_bytes;
    if (pr_block) *pr_block = g.block_bytes;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_server_submit_bfs(b2sr_server_t S, int32_t graph, int32_t src, int32_t* levels,
                                              int64_t* query_id) {
    clear_error();
    B2SR_TRY(check_server(S));
    if (!query_id || !levels) return fail(B2SR_ERR_INVALID_ARG, "levels or query_id is NULL");
    b2sr_matrix* h = nullptr;
    int64_t need = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (graph < 0 || graph >= (int32_t)S->graphs.size()) return fail(B2SR_ERR_INVALID_ARG, "no such graph");
        h = S->graphs[graph]->h;
        need = S->graphs[graph]->bfs_bytes;
    }
    if (src < 0 || src >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    if (S->max_lanes < 1) return fail(B2SR_ERR_ADMISSION_REFUSED, "no BFS lanes");
    auto* q = new QueryRec();
    q->kind = 0;
    q->graph = graph;
    q->src = src;
    q->out = levels;
    return enqueue(S, q, need, query_id);
}

extern "C" b2sr_status b2sr_server_submit_pagerank(b2sr_server_t S, int32_t graph, int32_t src, float d, int iters,
                                                   float* pr, int64_t* query_id) {
    clear_error();
    B2SR_TRY(check_server(S));
    if (!query_id || !pr) return fail(B2SR_ERR_INVALID_ARG, "pr or query_id is NULL");
    if (iters < 0 || !(d >= 0.0f && d <= 1.0f)) return fail(B2SR_ERR_INVALID_ARG, "bad iters or damping");
    b2sr_matrix* h = nullptr;
    int64_t need = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (graph < 0 || graph >= (int32_t)S->graphs.size()) return fail(B2SR_ERR_INVALID_ARG, "no such graph");
        h = S->graphs[graph]->h;
        need = S->graphs[graph]->block_bytes;
    }
    if (src >= h->n) return fail(B2SR_ERR_INVALID_ARG, "source out of range");
    if (h->n == 0) return fail(B2SR_ERR_INVALID_ARG, "empty graph");
    if (S->max_blocks < 1) return fail(B2SR_ERR_ADMISSION_REFUSED, "no PageRank blocks");
    auto* q = new QueryRec();
    q->kind = 1;
    q->graph = graph;
    q->src = src < 0 ? -1 : src;
    q->damp = d;
    q->iters = iters;
    q->out = pr;
    return enqueue(S, q, need, query_id);
}

extern "C" b2sr_status b2sr_server_wait(b2sr_server_t S, int64_t query_id, double timeout_s, int* done,
                                        double* latency_us) {
    clear_error();
    B2SR_TRY(check_server(S));
    if (!done) return fail(B2SR_ERR_INVALID_ARG, "done is NULL");
    *done = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->queries.find(query_id);
    if (it == S->queries.end()) return fail(B2SR_ERR_INVALID_ARG, "no such query");
    QueryRec* q = it->second.get();
    auto ready = [&] { return q->state.load() >= Q_DONE; };
    if (timeout_s > 0) S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    if (!ready()) return B2SR_OK;
    *done = 1;
    if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(q->t_done - q->t_submit).count();
    if (q->state.load() == Q_FAILED) return fail(q->status, "query failed: " + S->worker_error);
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_server_drain(b2sr_server_t S, double timeout_s) {
    clear_error();
    B2SR_TRY(check_server(S));
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9),
                                        [&] { return S->outstanding == 0; });
    if (!ok) return fail(B2SR_ERR_NOT_CONVERGED, "queries still outstanding at the timeout");
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_server_stats(b2sr_server_t S, b2sr_server_stats_t* out) {
    clear_error();
    B2SR_TRY(check_server(S));
    if (!out) return fail(B2SR_ERR_INVALID_ARG, "out is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = b2sr_server_stats_t{};
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->refused = S->refused;
    out->steps = S->steps;
    out->bytes_in_use = S->used;
    out->budget = S->budget;
    std::vector<double> l = S->lat_us;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {  // nearest rank
            size_t r = (size_t)std::ceil(p / 100.0 * (double)l.size());
            return l[std::min(l.size() - 1, r > 0 ? r - 1 : 0)];
        };
        out->p50_us = pct(50.0);
        out->p99_us = pct(99.0);
        out->max_us = l.back();
        double s = 0.0;
        for (double v : l) s += v;
        out->mean_us = s / (double)l.size();
    }
    if (S->have_t0 && S->completed > 0) {
        out->wall_s = std::chrono::duration<double>(S->t_last - S->t0).count();
        out->queries_per_s = out->wall_s > 0 ? (double)S->completed / out->wall_s : 0.0;
    }
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_server_reset_stats(b2sr_server_t S) {
    clear_error();
    B2SR_TRY(check_server(S));
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_us.clear();
    S->submitted = S->completed = S->failed = S->refused = S->steps = 0;
    S->have_t0 = false;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_server_destroy(b2sr_server_t S) {
    clear_error();
    if (!S) return B2SR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    while (!S->inbox.empty()) {  // queries never routed to a graph
        b2sr::QueryRec* q = S->inbox.front();
        S->inbox.pop_front();
        q->status = B2SR_ERR_ABORTED;
        q->state.store(b2sr::Q_FAILED);
    }
    for (auto& g : S->graphs) {
        if (g->found_host) cudaFreeHost(g->found_host);
        if (g->ev) cudaEventDestroy(g->ev);
        if (g->st) cudaStreamDestroy(g->st);
    }
    delete S;
    return B2SR_OK;
}
