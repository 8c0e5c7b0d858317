// zc_tune.cu -- CUDA graphs of zc calls and the autotuner of batched
// compression.  Both sit on top of the public C ABI (include/zc.h).
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "zc.h"

struct zc_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

int zc_graph_begin(zc_stream_t s)
{
    if (s == nullptr) return ZC_ERR_ARG;  // the legacy default stream cannot be captured
    return cudaStreamBeginCapture((cudaStream_t)s, cudaStreamCaptureModeThreadLocal) == cudaSuccess
               ? ZC_OK
               : ZC_ERR_CUDA;
}

int zc_graph_end(zc_stream_t s, zc_graph* g)
{
    if (s == nullptr || g == nullptr) return ZC_ERR_ARG;
    *g = nullptr;
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture((cudaStream_t)s, &graph) != cudaSuccess || graph == nullptr)
        return ZC_ERR_CUDA;
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return ZC_ERR_CUDA;
    }
    zc_graph_s* h = new zc_graph_s{graph, exec};
    *g = h;
    return ZC_OK;
}

int zc_graph_launch(zc_graph g, zc_stream_t s)
{
    if (g == nullptr) return ZC_ERR_ARG;
    return cudaGraphLaunch(g->exec, (cudaStream_t)s) == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

void zc_graph_destroy(zc_graph g)
{
    if (g == nullptr) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}

int zc_autotune_batch(int n_msgs, const zc_message* h_msgs, int tune_block, double link_gbs,
                      int reps, void* d_packed, size_t packed_cap, uint64_t* d_msg_off,
                      void* d_table, size_t table_bytes, void* d_ws, size_t ws_bytes,
                      zc_stream_t s, zc_tune_point* h_points, int max_points, int* n_points,
                      zc_tune_point* best)
{
    if (n_msgs < 1 || h_msgs == nullptr || best == nullptr || reps < 1 || reps > 100 ||
        d_msg_off == nullptr || d_ws == nullptr)
        return ZC_ERR_ARG;
    if (n_points) *n_points = 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return ZC_ERR_CUDA;
    const cudaStream_t cs = (cudaStream_t)s;

    std::vector<int> blocks;
    if (tune_block) blocks = {16, 32, 64, 128};
    else blocks = {0};
    const int chunk_opts[3] = {4, 8, 16};
    const int grid_opts[4] = {sms, 2 * sms, 4 * sms, 0};

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return ZC_ERR_CUDA;
    }
    std::vector<zc_message> msgs(h_msgs, h_msgs + n_msgs);
    std::vector<zc_tune_point> pts;
    int rc = ZC_OK;
    bool have_best = false;
    for (int blk : blocks) {
        for (int i = 0; i < n_msgs; ++i)
            msgs[(size_t)i].block = (blk == 0 || h_msgs[i].block == ZC_RAW) ? h_msgs[i].block : blk;
        for (int C : chunk_opts) {
            for (int G : grid_opts) {
                zc_batch plan;
                int st = zc_plan_compress_batch(&plan, n_msgs, msgs.data(), C, G, d_packed,
                                                packed_cap, d_msg_off, d_table, table_bytes);
                if (st) {
                    rc = st;
                    goto done;
                }
                if (G > 0 && (uint64_t)G >= plan.total_tiles) continue;  // same as grid 0
                zc_tune_point p;
                std::memset(&p, 0, sizeof(p));
                p.block = blk;
                p.tile_chunks = C;
                p.grid = G;
                if (zc_clear_device_status(d_ws, s) || zc_compress_batch(&plan, d_ws, ws_bytes, s)) {
                    rc = ZC_ERR_CUDA;
                    goto done;
                }
                std::vector<float> t((size_t)reps);
                for (int r = 0; r < reps && rc == ZC_OK; ++r) {
                    if (cudaEventRecord(e0, cs) != cudaSuccess ||
                        zc_compress_batch(&plan, d_ws, ws_bytes, s) != ZC_OK ||
                        cudaEventRecord(e1, cs) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&t[(size_t)r], e0, e1) != cudaSuccess)
                        rc = ZC_ERR_CUDA;
                }
                if (rc) goto done;
                std::sort(t.begin(), t.end());
                p.ms = t[t.size() / 2];
                uint64_t total = 0;
                if (cudaMemcpy(&total, d_msg_off + n_msgs, sizeof(total), cudaMemcpyDeviceToHost) !=
                    cudaSuccess) {
                    rc = ZC_ERR_CUDA;
                    goto done;
                }
                uint64_t detail = 0;
                if (zc_get_device_status(d_ws, s, &p.status, &detail)) {
                    rc = ZC_ERR_CUDA;
                    goto done;
                }
                p.packed_bytes = total;
                p.score_ms = p.ms + (link_gbs > 0.0 ? (double)total / (link_gbs * 1e6) : 0.0);
                pts.push_back(p);
                if (p.status == ZC_OK && (!have_best || p.score_ms < best->score_ms)) {
                    *best = p;
                    have_best = true;
                }
            }
        }
    }
    if (!have_best) {
        rc = pts.empty() ? ZC_ERR_ARG : pts.front().status;
        goto done;
    }
    // leave the table planned with the winner
    for (int i = 0; i < n_msgs; ++i)
        msgs[(size_t)i].block =
            (best->block == 0 || h_msgs[i].block == ZC_RAW) ? h_msgs[i].block : best->block;
    {
        zc_batch plan;
        rc = zc_plan_compress_batch(&plan, n_msgs, msgs.data(), best->tile_chunks, best->grid,
                                    d_packed, packed_cap, d_msg_off, d_table, table_bytes);
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h_points && max_points > 0) {
        const int k = std::min(max_points, (int)pts.size());
        for (int i = 0; i < k; ++i) h_points[i] = pts[(size_t)i];
    }
    if (n_points) *n_points = (int)pts.size();
    return rc;
}

}  // extern "C"
