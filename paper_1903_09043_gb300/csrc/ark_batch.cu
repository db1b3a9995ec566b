// ark_batch.cu -- ensembles of independent 2D runs advanced by one launch per
// step (ark_batch_* in include/ark.h).
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ark_handle.h"
#include "ark_step.cuh"

struct ark_batch {
    int count = 0, prec = 0, visc = 0;
    cudaStream_t stream = nullptr;
    std::vector<ark_handle*> runs;
    int nsm = 152;
    // launch configuration
    int tx = 0, width = 0, planes = 0;   // output tile width, kernel row width, planes per item
    ark::BatchKernelInfo kinfo{};
    int blocks = 0, nitems = 0;
    ark::StepArgs* d_args = nullptr;   // [6 phases][count]
    ark::BatchItem* d_items = nullptr;
    int* d_ctr = nullptr;              // 3 work counters (step % 3) + 3 for tuning
    void* d_scratch = nullptr;         // control words of tuning launches
    cudaGraphExec_t graph = nullptr;
    long long step = 0;
    std::string err;
};

namespace {

ark_status bfail(ark_batch* b, ark_status s, const std::string& m)
{
    if (b) b->err = m;
    return s;
}

#define BCUDA(b, call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return bfail((b), ARK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void drop_graph(ark_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// Work items and per-phase argument arrays for the kernel instance of row
// width `width` (its output tile width is kinfo.tx) and `planes` planes per
// item.  Phase p (= step % 6): input buffer p % 2, output the other,
// time-step slots read p % 3, write (p + 1) % 3, reset (p + 2) % 3.
ark_status configure(ark_batch* b, int width, int planes)
{
    ark::BatchKernelInfo k = ark::batch_kernel_2d(b->prec, b->visc, width);
    const int tx = k.tx;
    if (!k.func) return bfail(b, ARK_ERR_UNSUPPORTED, "no batched kernel for this precision / tile width");
    BCUDA(b, cudaFuncSetAttribute(k.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    int per_sm = 0;
    BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.func, k.threads, k.smem));
    if (per_sm < 1) return bfail(b, ARK_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
    std::vector<ark::BatchItem> items;
    std::vector<ark::StepArgs> args(6 * (size_t)b->count);
    for (int r = 0; r < b->count; ++r) {
        ark_handle* h = b->runs[r];
        const int nx = h->p.grid.n[0], ny = h->p.grid.n[1];
        const int tiles = (nx + tx - 1) / tx, chunks = (ny + planes - 1) / planes;
        for (int c = 0; c < chunks; ++c)
            for (int t = 0; t < tiles; ++t) items.push_back(ark::BatchItem{r, t, c, 0});
        ark::StepArgs a = ark::base_args(h);
        a.planes = planes;
        a.tiles_x = tiles;
        a.tiles_y = 1;
        a.dt_fixed = 0.0;
        for (int p = 0; p < 6; ++p) {
            ark::StepArgs ap = a;
            ap.Uin = h->U[p % 2];
            ap.Uout = h->U[(p + 1) % 2];
            ap.slot_read = p % 3;
            ap.slot_write = (p + 1) % 3;
            ap.slot_reset = (p + 2) % 3;
            args[(size_t)p * b->count + r] = ap;
        }
    }
    drop_graph(b);
    cudaFree(b->d_args);
    cudaFree(b->d_items);
    b->d_args = nullptr;
    b->d_items = nullptr;
    BCUDA(b, cudaMalloc(&b->d_args, args.size() * sizeof(ark::StepArgs)));
    BCUDA(b, cudaMalloc(&b->d_items, items.size() * sizeof(ark::BatchItem)));
    BCUDA(b, cudaMemcpyAsync(b->d_args, args.data(), args.size() * sizeof(ark::StepArgs), cudaMemcpyHostToDevice, b->stream));
    BCUDA(b, cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(ark::BatchItem), cudaMemcpyHostToDevice,
                             b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));   // host vectors leave scope
    b->kinfo = k;
    b->tx = tx;
    b->width = width;
    b->planes = planes;
    b->nitems = (int)items.size();
    b->blocks = per_sm * b->nsm;
    if (b->blocks > b->nitems) b->blocks = b->nitems;
    return ARK_OK;
}

ark_status launch_phase(ark_batch* b, const ark::StepArgs* runs, int ctr_base, int ctr_cur, int ctr_next)
{
    const ark::BatchItem* items = b->d_items;
    int nitems = b->nitems;
    int* ctr = b->d_ctr + ctr_base;
    void* params[] = {(void*)&runs, (void*)&items, (void*)&nitems, (void*)&ctr, (void*)&ctr_cur, (void*)&ctr_next};
    BCUDA(b, cudaLaunchKernel(b->kinfo.func, dim3(b->blocks), dim3(b->kinfo.threads), params, b->kinfo.smem, b->stream));
    return ARK_OK;
}

// One graph of the six phases of a cycle, chained.
ark_status build_graph(ark_batch* b)
{
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaGraphCreate(&g, 0));
    cudaGraphNode_t prev = nullptr;
    const ark::BatchItem* items = b->d_items;
    int nitems = b->nitems;
    int* ctr = b->d_ctr;
    ark_status st = ARK_OK;
    for (int p = 0; p < 6 && st == ARK_OK; ++p) {
        const ark::StepArgs* runs = b->d_args + (size_t)p * b->count;
        int cur = p % 3, next = (p + 1) % 3;
        void* params[] = {(void*)&runs, (void*)&items, (void*)&nitems, (void*)&ctr, (void*)&cur, (void*)&next};
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof kp);
        kp.func = const_cast<void*>(b->kinfo.func);
        kp.gridDim = dim3(b->blocks);
        kp.blockDim = dim3(b->kinfo.threads);
        kp.sharedMemBytes = (unsigned)b->kinfo.smem;
        kp.kernelParams = params;
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        if (e != cudaSuccess) st = bfail(b, ARK_ERR_CUDA, std::string("cudaGraphAddKernelNode: ") + cudaGetErrorString(e));
        prev = node;
    }
    if (st == ARK_OK) {
        cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
        if (e != cudaSuccess) st = bfail(b, ARK_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    cudaGraphDestroy(g);
    return st;
}

ark_status check_run(ark_batch* b, int run)
{
    if (!b) return ARK_ERR_INVALID_ARG;
    if (run < 0 || run >= b->count) return bfail(b, ARK_ERR_INVALID_ARG, "run index out of range");
    return ARK_OK;
}

ark_status from_run(ark_batch* b, ark_handle* h, ark_status st)
{
    if (st != ARK_OK) b->err = h->err;
    return st;
}

}  // namespace

extern "C" {

ark_status ark_batch_create(int count, const ark_params* params, void* cuda_stream, ark_batch** out)
{
    if (!out || !params || count < 1) return ARK_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        const ark_params& p = params[i];
        if (p.grid.dim != 2) return ARK_ERR_UNSUPPORTED;
        if (p.precision != params[0].precision) return ARK_ERR_INVALID_ARG;
        if (p.precision == ARK_F32) return ARK_ERR_UNSUPPORTED;
        if (p.gravity.phi) return ARK_ERR_UNSUPPORTED;   // ensembles take uniform gravity
        if (p.eos.law != ARK_EOS_STIFFENED_GAS) return ARK_ERR_UNSUPPORTED;   // and the stiffened gas
        if (p.bc.lo[0] == ARK_BC_HALO || p.bc.hi[0] == ARK_BC_HALO) return ARK_ERR_UNSUPPORTED;   // whole grids
        if ((p.mu > 0.0 || p.kappa > 0.0) != (params[0].mu > 0.0 || params[0].kappa > 0.0)) return ARK_ERR_INVALID_ARG;
    }
    ark_batch* b = new (std::nothrow) ark_batch();
    if (!b) return ARK_ERR_ALLOC;
    b->count = count;
    b->prec = params[0].precision;
    b->visc = (params[0].mu > 0.0 || params[0].kappa > 0.0) ? 1 : 0;
    b->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete b;
        return ARK_ERR_CUDA;
    }
    for (int i = 0; i < count; ++i) {
        ark_handle* h = nullptr;
        ark_status st = ark_create(&params[i], cuda_stream, &h);
        if (st != ARK_OK) {
            ark_batch_destroy(b);
            return st;
        }
        b->runs.push_back(h);
    }
    if (cudaMalloc(&b->d_ctr, 8 * sizeof(int)) != cudaSuccess || cudaMalloc(&b->d_scratch, 256) != cudaSuccess ||
        cudaMemsetAsync(b->d_ctr, 0, 8 * sizeof(int), b->stream) != cudaSuccess) {
        cudaGetLastError();
        ark_batch_destroy(b);
        return ARK_ERR_ALLOC;
    }
    *out = b;
    return ARK_OK;
}

ark_status ark_batch_destroy(ark_batch* b)
{
    if (!b) return ARK_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (ark_handle* h : b->runs) ark_destroy(h);
    cudaFree(b->d_args);
    cudaFree(b->d_items);
    cudaFree(b->d_ctr);
    cudaFree(b->d_scratch);
    delete b;
    return ARK_OK;
}

ark_status ark_batch_set_state(ark_batch* b, int run, const double* U, int on_device)
{
    ark_status st = check_run(b, run);
    if (st != ARK_OK) return st;
    return from_run(b, b->runs[run], ark_set_state(b->runs[run], U, on_device));
}

ark_status ark_batch_get_state(ark_batch* b, int run, double* U, int on_device)
{
    ark_status st = check_run(b, run);
    if (st != ARK_OK) return st;
    return from_run(b, b->runs[run], ark_get_state(b->runs[run], U, on_device));
}

ark_status ark_batch_diagnostics(ark_batch* b, int run, ark_diag* out)
{
    ark_status st = check_run(b, run);
    if (st != ARK_OK) return st;
    return from_run(b, b->runs[run], ark_diagnostics(b->runs[run], out));
}

ark_status ark_batch_tune(ark_batch* b, int reps, int* tx_out, int* planes_out)
{
    if (!b || reps < 1) return ARK_ERR_INVALID_ARG;
    for (ark_handle* h : b->runs)
        if (!h->state_set) return bfail(b, ARK_ERR_INVALID_ARG, "tune needs every run's state");
    const int txs[3] = {64, 128, 256}, pls[3] = {16, 32, 64};
    float best = 1e30f;
    int btx = 0, bpl = 0;
    cudaEvent_t e0, e1;
    BCUDA(b, cudaEventCreate(&e0));
    BCUDA(b, cudaEventCreate(&e1));
    ark_status st = ARK_OK;
    for (int i = 0; i < 3 && st == ARK_OK; ++i)
        for (int j = 0; j < 3 && st == ARK_OK; ++j) {
            st = configure(b, txs[i], pls[j]);
            if (st == ARK_OK) {
                // tuning arguments: read the current states, write the spare buffers,
                // fixed tiny dt, time / slots / status redirected to scratch
                std::vector<ark::StepArgs> args((size_t)b->count);
                for (int r = 0; r < b->count; ++r) {
                    ark_handle* h = b->runs[r];
                    ark::StepArgs a = ark::base_args(h);
                    a.planes = b->planes;
                    a.tiles_x = (h->p.grid.n[0] + b->tx - 1) / b->tx;
                    a.tiles_y = 1;
                    a.Uin = h->U[h->cur];
                    a.Uout = h->U[1 - h->cur];
                    a.dt_fixed = 1e-12;
                    char* sc = (char*)b->d_scratch;
                    a.smax = (unsigned long long*)sc;
                    a.status = (unsigned int*)(sc + 32);
                    a.time = (double*)(sc + 64);
                    a.dt_last = (double*)(sc + 72);
                    a.slot_read = 0;
                    a.slot_write = 1;
                    a.slot_reset = 2;
                    args[r] = a;
                }
                // phase-0 slice of d_args is reused for the tuning arguments
                cudaError_t e = cudaMemcpyAsync(b->d_args, args.data(), args.size() * sizeof(ark::StepArgs),
                                                cudaMemcpyHostToDevice, b->stream);
                if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctr + 3, 0, 3 * sizeof(int), b->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
                if (e != cudaSuccess) st = bfail(b, ARK_ERR_CUDA, cudaGetErrorString(e));
                for (int k = 0; k <= reps && st == ARK_OK; ++k) {
                    if (k == 1) cudaEventRecord(e0, b->stream);
                    st = launch_phase(b, b->d_args, 3, k % 3, (k + 1) % 3);
                }
                if (st == ARK_OK) {
                    cudaEventRecord(e1, b->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) { best = ms; btx = txs[i]; bpl = pls[j]; }
                }
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != ARK_OK) return st;
    st = configure(b, btx, bpl);   // rebuilds the real argument arrays
    if (st != ARK_OK) return st;
    if (tx_out) *tx_out = b->tx;
    if (planes_out) *planes_out = bpl;
    return ARK_OK;
}

ark_status ark_batch_step(ark_batch* b, int nsteps)
{
    if (!b || nsteps < 0) return ARK_ERR_INVALID_ARG;
    for (ark_handle* h : b->runs) {
        if (!h->state_set) return bfail(b, ARK_ERR_INVALID_ARG, "every run needs a state");
        if (h->step != b->step || h->cur != (int)(b->step % 2))
            return bfail(b, ARK_ERR_INVALID_ARG, "runs out of lockstep (a run was reloaded after stepping)");
    }
    if (nsteps == 0) return ARK_OK;
    if (!b->kinfo.func) {
        // untuned default: tile width close to the typical run width, 32 planes per item
        ark_status st = configure(b, 128, 32);
        if (st != ARK_OK) return st;
    }
    for (ark_handle* h : b->runs) {
        ark_status st = ark::ensure_dt(h);
        if (st != ARK_OK) return from_run(b, h, st);
    }
    while (nsteps > 0) {
        const int p = (int)(b->step % 6);
        if (p == 0 && nsteps >= 6) {
            if (!b->graph) {
                ark_status st = build_graph(b);
                if (st != ARK_OK) return st;
            }
            BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
            b->step += 6;
            nsteps -= 6;
        } else {
            ark_status st = launch_phase(b, b->d_args + (size_t)p * b->count, 0, p % 3, (p + 1) % 3);
            if (st != ARK_OK) return st;
            b->step += 1;
            nsteps -= 1;
        }
    }
    for (ark_handle* h : b->runs) {
        h->step = b->step;
        h->cur = (int)(b->step % 2);
        h->dt_valid = true;
    }
    return ARK_OK;
}

ark_status ark_batch_shape(const ark_batch* b, int* tx, int* planes, int* items, int* blocks)
{
    if (!b) return ARK_ERR_INVALID_ARG;
    if (tx) *tx = b->tx;
    if (planes) *planes = b->planes;
    if (items) *items = b->nitems;
    if (blocks) *blocks = b->blocks;
    return ARK_OK;
}

const char* ark_batch_last_error(const ark_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
