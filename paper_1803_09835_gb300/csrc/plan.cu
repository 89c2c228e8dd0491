// plan.cu -- batched search plans: a fixed batch shape (stations and their
// lengths) whose table build runs as one captured CUDA graph, and whose
// search options are picked by a small autotuner on the first run.
//
// Creation traces one build to size a device arena, then captures the build
// -- the signature launch, the radix passes (4 key passes + the station
// pass), the occurrence filter -- into a graph with every buffer inside the
// arena, so replays allocate nothing.  The first run times the search under
// each candidate option set (vote path, dense-group threshold, row-group size,
// map load) and keeps the fastest; every option set gives the same detections.
#include <algorithm>

#include "fast_internal.cuh"

using namespace fastgb;

struct fast_plan {
    fast_ctx *c = nullptr;
    std::vector<uint64_t> soff;
    uint64_t N = 0;
    uint32_t ld = 0;
    const uint16_t *d_idx = nullptr;
    char *arena = nullptr;
    uint64_t arena_size = 0;
    uint32_t *sig = nullptr;
    fast_tables *tb = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_nodes = 0, graph_kernels = 0;
    float build_ms = 0.f;  // the last replay of the build graph (with the timing option)
    bool tuned = false;
    fast_plan_choice best{};
    std::vector<fast_plan_choice> tried;
};

namespace {

fast_status apply(fast_ctx *c, const fast_plan_choice &o) {
    c->vote_map = o.vote_map != 0;
    c->large_min = o.large_min;
    c->map_load = o.map_load;
    c->group_pairs = o.group_pairs;
    return FAST_OK;
}

// the graph's build, also used (untraced) to size the arena
fast_status plan_build(fast_plan *P, cudaStream_t s) {
    fast_ctx *c = P->c;
    const size_t n = (size_t)c->p.b * P->N;
    fast_status st = dalloc_t(c, &P->sig, n ? n : 1, s);
    if (st) return st;
    if ((st = sig_launch(c, P->d_idx, P->N, P->ld, P->sig, s))) return st;
    return build_tables(c, P->sig, P->N, P->soff.data(), (uint32_t)P->soff.size() - 1, &P->tb, s);
}

}  // namespace

extern "C" {

fast_status fast_plan_create(fast_ctx *c, const uint16_t *d_idx, const uint64_t *h_station_N, uint32_t n_st,
                             uint32_t ld, void *stream, fast_plan **out) {
    if (!c || !out || !h_station_N || n_st == 0 || n_st > 256 || ld < c->p.K) return FAST_EINVAL;
    *out = nullptr;
    c->err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return set_error(c, FAST_EINVAL, "plans need a non-default stream (graph capture)");
    fast_plan *P = new fast_plan();
    P->c = c;
    P->ld = ld;
    P->d_idx = d_idx;
    P->soff.assign(n_st + 1, 0);
    for (uint32_t x = 0; x < n_st; x++) P->soff[x + 1] = P->soff[x] + h_station_N[x];
    P->N = P->soff[n_st];
    if (P->N == 0 || P->N > (1ull << 28) - 1 || !d_idx) {
        delete P;
        return set_error(c, FAST_EINVAL, "plan needs 1 .. 2^28 - 1 windows");
    }
    // 1. trace one ordinary build to learn the arena size
    c->trace = true;
    c->trace_total = 0;
    fast_status st = plan_build(P, s);
    c->trace = false;
    if (P->tb) fast_tables_free(P->tb);
    P->tb = nullptr;
    dfree(c, P->sig, (size_t)c->p.b * P->N * 4, s);
    P->sig = nullptr;
    if (!st) st = sync_check(c, s, "plan trace");
    if (st) {
        delete P;
        return st;
    }
    P->arena_size = c->trace_total + (1 << 20);
    if (c->budget && c->live + P->arena_size > c->budget) {
        delete P;
        return set_error(c, FAST_EBUDGET, "plan arena does not fit the HBM budget");
    }
    cudaError_t e = cudaMalloc(&P->arena, P->arena_size);
    if (e) {
        delete P;
        return cuda_fail(c, e, "plan arena");
    }
    c->live += P->arena_size;
    // 2. capture the build into a graph, every buffer in the arena
    c->arena = P->arena;
    c->arena_size = P->arena_size;
    c->arena_off = 0;
    c->capturing = true;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (!e) {
        st = plan_build(P, s);
        e = cudaStreamEndCapture(s, &P->graph);
    }
    c->capturing = false;
    c->arena = nullptr;
    if (!st && e) st = cuda_fail(c, e, "graph capture");
    if (!st && (e = cudaGraphInstantiate(&P->exec, P->graph, 0))) st = cuda_fail(c, e, "graph instantiate");
    if (!st) {
        cudaGraphGetNodes(P->graph, nullptr, &P->graph_nodes);
        std::vector<cudaGraphNode_t> nodes(P->graph_nodes);
        if (P->graph_nodes) cudaGraphGetNodes(P->graph, nodes.data(), &P->graph_nodes);
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) P->graph_kernels++;
        }
        cudaMemcpy(P->tb->d_soff, P->soff.data(), P->soff.size() * 8, cudaMemcpyHostToDevice);
    }
    if (st) {
        fast_plan_destroy(P);
        return st;
    }
    *out = P;
    return FAST_OK;
}

void fast_plan_destroy(fast_plan *P) {
    if (!P) return;
    fast_ctx *c = P->c;
    cudaDeviceSynchronize();
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    delete P->tb;  // its buffers live in the arena
    if (P->arena) {
        cudaFree(P->arena);
        c->live -= std::min<uint64_t>(c->live, P->arena_size);
    }
    cudaGetLastError();
    delete P;
}

static fast_status plan_run(fast_plan *P, fast_result **out, cudaStream_t s);

fast_status fast_plan_run(fast_plan *P, fast_result **out, void *stream) {
    if (!P || !out) return FAST_EINVAL;
    fast_ctx *c = P->c;
    // the context's own options come back after the run
    const fast_plan_choice saved{c->vote_map ? 1u : 0u, c->large_min, c->map_load, 0.f, c->group_pairs};
    const fast_status st = plan_run(P, out, (cudaStream_t)stream);
    apply(c, saved);
    return st;
}

}  // extern "C"

static fast_status plan_run(fast_plan *P, fast_result **out, cudaStream_t s) {
    fast_ctx *c = P->c;
    c->err.clear();
    const uint32_t n_st = (uint32_t)P->soff.size() - 1;
    for (uint32_t x = 0; x < n_st; x++) out[x] = nullptr;
    stage_reset();
    c->stats.n_launches = 0;
    stage_mark(c, 0, s);
    cudaError_t e = cudaGraphLaunch(P->exec, s);
    if (e) return cuda_fail(c, e, "graph launch");
    stage_mark(c, 9, s);
    // the filter's drop count, left in the device counters by the graph
    cudaMemcpyAsync(c->h_scal + Scal::NDROP, c->d_scal + Scal::NDROP, 8, cudaMemcpyDeviceToHost, s);
    fast_status st = sync_check(c, s, "plan build");
    if (st) return st;
    P->tb->n_dropped = c->h_scal[Scal::NDROP];
    P->build_ms = stage_ms(c, 0, 9);
    const uint64_t graph_launches = P->graph_kernels;
    fast_result *all = nullptr;
    if (!P->tuned) {
        c->large_min = 0;
        const uint32_t lm = large_min_for(c, P->N);
        const fast_plan_choice cand[] = {{0, 0, 0.5f, 0.f, 0},      {0, 0, 0.5f, 0.f, 512},   {0, 0, 0.5f, 0.f, 2048},
                                         {0, 2 * lm, 0.5f, 0.f, 0}, {0, 8 * lm, 0.5f, 0.f, 0}, {1, 0, 0.5f, 0.f, 0},
                                         {1, 0, 0.85f, 0.f, 0}};
        float best_ms = 1e30f;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        for (const fast_plan_choice &o : cand) {
            apply(c, o);
            cudaEventRecord(a, s);
            fast_result *r = nullptr;
            st = search_run(c, P->tb, P->sig, &r, s);
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            if (st) break;
            fast_plan_choice tr = o;
            cudaEventElapsedTime(&tr.ms, a, b);
            P->tried.push_back(tr);
            if (tr.ms < best_ms) {
                best_ms = tr.ms;
                P->best = tr;
                fast_result_free(all);
                all = r;
            } else {
                fast_result_free(r);
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (st) {
            fast_result_free(all);
            return st;
        }
        P->tuned = true;
        apply(c, P->best);
    } else {
        apply(c, P->best);
        if ((st = search_run(c, P->tb, P->sig, &all, s))) return st;
    }
    stage_mark(c, 8, s);
    if ((st = split_stations(c, all, P->soff, out, s))) return st;
    stats_times(c, true);
    c->stats.n_fingerprints = P->N;
    c->stats.n_launches += graph_launches;
    return FAST_OK;
}

extern "C" {

fast_status fast_plan_info(const fast_plan *P, fast_plan_info_t *info) {
    if (!P || !info) return FAST_EINVAL;
    info->graph_nodes = P->graph_nodes;
    info->graph_kernels = P->graph_kernels;
    info->build_ms = P->build_ms;
    info->arena_bytes = P->arena_size;
    info->tuned = P->tuned;
    info->best = P->best;
    info->n_tried = (uint32_t)std::min<size_t>(P->tried.size(), 8);
    for (uint32_t k = 0; k < info->n_tried; k++) info->tried[k] = P->tried[k];
    return FAST_OK;
}

}  // extern "C"
