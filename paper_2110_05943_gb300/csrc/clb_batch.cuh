// clb_batch.cuh -- batches of independent simulations advanced by one
// launch per step (host side of clb_batch_*; included by clb_api.cu).
//
// Each case is an ordinary clb_handle (its own buffers, parameters and
// reductions); the batch builds a device table of the cases and a tile list
// over the active ones and advances all of them, in one of two modes:
//   CLB_BATCH_GRAPH      : one launch per step -- k_step_batch for FP64,
//                          k_step_batch_mix for the FP16 forms (blocks of
//                          interior-pair tiles and blocks of edge nodes in
//                          one grid) -- replayed from CUDA graphs of
//                          kGraphSteps steps;
//   CLB_BATCH_PERSISTENT : one cooperative k_step_batch_persist launch per
//                          kGraphSteps steps (itself captured in a graph),
//                          its steps separated by a bounded grid barrier.
// Cases can be retired (e.g. once steady) and the tile shape is chosen by a
// measured sweep.

struct clb_batch {
    std::vector<clb_handle*> cases;
    std::vector<int32_t> active;
    std::vector<int32_t> flip;      // case c's current buffer is (par ^ flip[c]) while it is active
    int prec = CLB_F64;
    int shift = 1, forch = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_side = nullptr;  // graph capture: the edge kernel's branch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    void* table = nullptr;          // CaseT array on the device
    int4* tiles = nullptr;          // tile list on the device (all tiles; FP64 and the persistent mode)
    int ntiles = 0;
    int4* itiles = nullptr;         // FP16 forms, graph mode: interior-pair tiles (case, x0, y0)
    int n_itiles = 0;
    int4* echunks = nullptr;        // and chunks of edge nodes (case, first edge index, count)
    int n_echunks = 0;
    int4* work = nullptr;           // FP16 forms, one-launch steps: per block (0, first tile) or (1, edge chunk)
    int n_work = 0;
    int64_t nodes = 0;              // active nodes per step
    int par = 0;
    int64_t t = 0;
    int shape = 0;                  // index into kShapes
    int per_cta = 8;                // tiles per CTA
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_failed = false;
    int mode = CLB_BATCH_GRAPH;   // measured faster on the 512-case workload (FP16N 30.8 vs 30.1 GLUPS)
    GridBarrier* bar = nullptr;     // persistent mode: grid barrier state (device)
    int pgrid = 0;                  // persistent mode: resident blocks of the launch
    long long wait_limit = 4000000000LL;   // barrier wait bound, SM cycles (~2 s)
    std::string err;
};

namespace {
// Candidate block shapes (threads in x, threads in y), 128 threads each.
// Taller blocks reuse the pulled rows y - 1, y, y + 1 in L1 across their
// warps; wider ones waste less on narrow grids.
constexpr int kNumShapes = 4;
constexpr int kShapes[kNumShapes][2] = {{64, 2}, {32, 4}, {16, 8}, {8, 16}};
constexpr int kPerCta[3] = {4, 16, 64};
}  // namespace

static int bfail(clb_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_init_error = buf;
    return code;
}

#define CKB(b, call)                                                                                \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? CLB_ERR_OOM : CLB_ERR_CUDA,         \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                           \
    } while (0)

static void batch_drop_graphs(clb_batch* b) {
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
    b->graph_failed = false;
    b->pgrid = 0;
}

static int nodes_per_thread(const clb_batch* b) { return b->prec == CLB_F64 ? 1 : 2; }

// Uploads a host list (replacing *dev).
static int upload_list(clb_batch* b, const std::vector<int4>& host, int4** dev, int* n) {
    cudaFree(*dev);
    *dev = nullptr;
    *n = (int)host.size();
    if (*n) {
        CKB(b, cudaMalloc(dev, host.size() * sizeof(int4)));
        CKB(b, cudaMemcpy(*dev, host.data(), host.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    return CLB_OK;
}

// Tile lists over the active cases for the current block shape: all tiles
// (FP64, persistent mode) and, for the FP16 forms, the interior-pair tiles
// (pairs x0 = 2, 4, ... with x0 + 2 < nx, rows inside walled S/N sides) and
// the edge nodes in chunks of up to 128 (the same split as k_step2).
static int batch_build_tiles(clb_batch* b) {
    const int bx = kShapes[b->shape][0], by = kShapes[b->shape][1];
    const int tw = bx * nodes_per_thread(b);
    std::vector<int4> host, inner, edges;
    std::vector<long long> anchor;   // per edge chunk: the interior tile covering its last row (-1: none before)
    b->nodes = 0;
    for (size_t c = 0; c < b->cases.size(); ++c) {
        if (!b->active[c]) continue;
        const clb_params& p = b->cases[c]->prm;
        b->nodes += (int64_t)p.nx * p.ny;
        for (int y0 = 0; y0 < p.ny; y0 += by)
            for (int x0 = 0; x0 < p.nx; x0 += tw) host.push_back(make_int4((int)c, x0, y0, 0));
        if (b->prec == CLB_F64) continue;
        const Geo& G = b->cases[c]->k32.g;
        const int y_lo = G.wall_y ? 1 : 0, y_hi = G.wall_y ? G.ny - 2 : G.ny - 1;
        const long long first = (long long)inner.size();
        int ntx = 0, nty = 0;
        for (int y0 = y_lo; y0 <= y_hi; y0 += by, ++nty) {
            ntx = 0;
            for (int x0 = 2; x0 + 2 < G.nx; x0 += tw, ++ntx) inner.push_back(make_int4((int)c, x0, y0, 0));
        }
        const long long ne = edge_count(G);
        for (long long i0 = 0; i0 < ne; i0 += 128) {
            const int cnt = (int)std::min(128LL, ne - i0);
            edges.push_back(make_int4((int)c, (int)i0, cnt, 0));
            int ymax = 0;
            for (int k = 0; k < cnt; ++k) {
                int x, y;
                edge_node(G, i0 + k, x, y);
                ymax = std::max(ymax, y);
            }
            if (ntx == 0) {
                anchor.push_back(first - 1);
            } else {
                const int ty = std::min(std::max(ymax - y_lo, 0) / by, nty - 1);
                anchor.push_back(first + (long long)ty * ntx + ntx - 1);
            }
        }
    }
    // one-launch order: each interior block, then the edge chunks anchored in it
    std::vector<int4> work;
    if (b->prec != CLB_F64) {
        const int pc = b->per_cta;
        std::vector<std::vector<int>> after((inner.size() + pc - 1) / pc + 1);   // [0]: before every block
        for (size_t j = 0; j < edges.size(); ++j) after[anchor[j] < 0 ? 0 : anchor[j] / pc + 1].push_back((int)j);
        for (int j : after[0]) work.push_back(make_int4(1, j, 0, 0));
        for (size_t bi = 0; bi + 1 < after.size(); ++bi) {
            work.push_back(make_int4(0, (int)(bi * pc), 0, 0));
            for (int j : after[bi + 1]) work.push_back(make_int4(1, j, 0, 0));
        }
    }
    int rc = upload_list(b, host, &b->tiles, &b->ntiles);
    if (rc == CLB_OK) rc = upload_list(b, inner, &b->itiles, &b->n_itiles);
    if (rc == CLB_OK) rc = upload_list(b, edges, &b->echunks, &b->n_echunks);
    if (rc == CLB_OK) rc = upload_list(b, work, &b->work, &b->n_work);
    batch_drop_graphs(b);
    return rc;
}

// FP16 forms: interior tiles and edge chunks in one launch, each edge chunk
// after the interior block covering its rows (build-time option; 0 launches
// two kernels, which captured graphs run as parallel branches when
// CLB_BATCH_FORK is 1).
#ifndef CLB_BATCH_MIX
#define CLB_BATCH_MIX 1
#endif
#ifndef CLB_BATCH_FORK
#define CLB_BATCH_FORK 1
#endif

// One step.  With a side stream (graph capture) the edge kernel is a
// parallel branch beside the interior kernel -- they write disjoint nodes --
// so its few slow blocks run under the interior kernel instead of after it.
template <class P, int NPT>
static void batch_launch_as(clb_batch* b, cudaStream_t s, cudaStream_t side) {
    using C = CaseT<typename P::R, typename P::S>;
    const C* tab = (const C*)b->table;
    const dim3 block(kShapes[b->shape][0], kShapes[b->shape][1]);
    if constexpr (NPT == 2) {
        if (CLB_BATCH_MIX && b->n_work > 0) {
            const unsigned g = (unsigned)b->n_work;
            const int4 *w = b->work, *t = b->itiles, *e = b->echunks;
            const int n = b->n_itiles, pc = b->per_cta, par = b->par;
            if (b->shift && b->forch) k_step_batch_mix<P, true, true><<<g, block, 0, s>>>(tab, w, t, n, pc, e, par);
            else if (b->shift) k_step_batch_mix<P, true, false><<<g, block, 0, s>>>(tab, w, t, n, pc, e, par);
            else if (b->forch) k_step_batch_mix<P, false, true><<<g, block, 0, s>>>(tab, w, t, n, pc, e, par);
            else k_step_batch_mix<P, false, false><<<g, block, 0, s>>>(tab, w, t, n, pc, e, par);
            return;
        }
        const bool fork = side && b->n_itiles > 0 && b->n_echunks > 0;
        cudaStream_t es = s;
        if (fork && cudaEventRecord(b->ev_fork, s) == cudaSuccess && cudaStreamWaitEvent(side, b->ev_fork, 0) == cudaSuccess)
            es = side;
        if (b->n_echunks > 0) {
            const int4* e = b->echunks;
            const unsigned g = (unsigned)b->n_echunks;
            if (b->shift && b->forch) k_step_batch_edge<P, true, true><<<g, 128, 0, es>>>(tab, e, b->par);
            else if (b->shift) k_step_batch_edge<P, true, false><<<g, 128, 0, es>>>(tab, e, b->par);
            else if (b->forch) k_step_batch_edge<P, false, true><<<g, 128, 0, es>>>(tab, e, b->par);
            else k_step_batch_edge<P, false, false><<<g, 128, 0, es>>>(tab, e, b->par);
        }
        if (b->n_itiles > 0) {
            const int grid = (b->n_itiles + b->per_cta - 1) / b->per_cta;
            const int4* t = b->itiles;
            if (b->shift && b->forch) k_step_batch_int<P, true, true><<<grid, block, 0, s>>>(tab, t, b->n_itiles, b->per_cta, b->par);
            else if (b->shift) k_step_batch_int<P, true, false><<<grid, block, 0, s>>>(tab, t, b->n_itiles, b->per_cta, b->par);
            else if (b->forch) k_step_batch_int<P, false, true><<<grid, block, 0, s>>>(tab, t, b->n_itiles, b->per_cta, b->par);
            else k_step_batch_int<P, false, false><<<grid, block, 0, s>>>(tab, t, b->n_itiles, b->per_cta, b->par);
        }
        if (es != s) {   // join: the next step waits for both branches
            cudaEventRecord(b->ev_join, es);
            cudaStreamWaitEvent(s, b->ev_join, 0);
        }
    } else {
        const int grid = (b->ntiles + b->per_cta - 1) / b->per_cta;
        if (b->shift && b->forch) k_step_batch<P, NPT, true, true><<<grid, block, 0, s>>>(tab, b->tiles, b->ntiles, b->per_cta, b->par);
        else if (b->shift) k_step_batch<P, NPT, true, false><<<grid, block, 0, s>>>(tab, b->tiles, b->ntiles, b->per_cta, b->par);
        else if (b->forch) k_step_batch<P, NPT, false, true><<<grid, block, 0, s>>>(tab, b->tiles, b->ntiles, b->per_cta, b->par);
        else k_step_batch<P, NPT, false, false><<<grid, block, 0, s>>>(tab, b->tiles, b->ntiles, b->per_cta, b->par);
    }
}

// Persistent launch of `nsteps` steps from parity par0.  The grid is as
// many blocks as can be resident at once (cooperative launch), at most one
// per tile; the blocks claim the tuned number of tiles at a time.
template <class P, int NPT>
static cudaError_t batch_persist_as(clb_batch* b, cudaStream_t s, int par0, int nsteps, int extra,
                                    long long limit) {
    using C = CaseT<typename P::R, typename P::S>;
    using Fn = void (*)(const C*, const int4*, int, int, int, int, GridBarrier*, int, long long);
    Fn fn = b->shift ? (b->forch ? k_step_batch_persist<P, NPT, true, true> : k_step_batch_persist<P, NPT, true, false>)
                     : (b->forch ? k_step_batch_persist<P, NPT, false, true> : k_step_batch_persist<P, NPT, false, false>);
    const dim3 block(kShapes[b->shape][0], kShapes[b->shape][1]);
    if (b->pgrid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)(block.x * block.y), 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        b->pgrid = std::min(sms * per_sm, std::max(b->ntiles, 1));
    }
    const int chunk = b->per_cta;   // tiles claimed at a time (the tuned tiles per block)
    cudaError_t e = cudaMemsetAsync(b->bar, 0, offsetof(GridBarrier, failed), s);   // arrived, next[]
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)b->pgrid);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, (const C*)b->table, (const int4*)b->tiles, b->ntiles, chunk, par0, nsteps,
                              b->bar, extra, limit);
}

// Persistent launch in the batch's precision (coherent loads, see LdCA).
#ifndef CLB_PERSIST_LD
#define CLB_PERSIST_LD LdCA
#endif
static cudaError_t batch_persist(clb_batch* b, cudaStream_t s, int par0, int nsteps, int extra, long long limit) {
    using L = CLB_PERSIST_LD;
    if (b->ntiles == 0) return cudaSuccess;
    if (b->prec == CLB_F16S) return batch_persist_as<StoreH16T<L>, 2>(b, s, par0, nsteps, extra, limit);
    if (b->prec == CLB_F16N) return batch_persist_as<StoreH16NT<L>, 2>(b, s, par0, nsteps, extra, limit);
    return batch_persist_as<StoreF64T<L>, 1>(b, s, par0, nsteps, extra, limit);
}

static void batch_launch(clb_batch* b, cudaStream_t s, cudaStream_t side = nullptr) {
    if (b->ntiles > 0) {
        if (b->prec == CLB_F16S) batch_launch_as<StoreH16, 2>(b, s, side);
        else if (b->prec == CLB_F16N) batch_launch_as<StoreH16N, 2>(b, s, side);
        else batch_launch_as<StoreF64, 1>(b, s, side);
    }
    b->par = 1 - b->par;
}

static cudaGraphExec_t batch_capture(clb_batch* b, int par) {
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    const int save = b->par;
    b->par = par;
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        b->par = save;
        cudaGetLastError();
        return nullptr;
    }
    if (b->mode == CLB_BATCH_PERSISTENT) batch_persist(b, b->cap_stream, par, kGraphSteps, 0, b->wait_limit);
    else
        for (int i = 0; i < kGraphSteps; ++i) batch_launch(b, b->cap_stream, CLB_BATCH_FORK ? b->cap_side : nullptr);
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &gr);
    b->par = save;
    if (e != cudaSuccess || !gr) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) ex = nullptr;
    cudaGraphDestroy(gr);
    cudaGetLastError();
    return ex;
}

// Keep the active case handles' buffer parity in step with the batch; a
// retired case keeps the parity (the buffer) its state was left in.
static void batch_sync_cases(clb_batch* b) {
    for (size_t c = 0; c < b->cases.size(); ++c)
        if (b->active[c]) b->cases[c]->par = b->par ^ b->flip[c];
}

// Device copy of case c's flip in the case table.
static int batch_upload_flip(clb_batch* b, size_t c) {
    using C64 = CaseT<double, double>;
    using C16 = CaseT<float, __half>;
    size_t off, stride;
    if (b->prec == CLB_F64) {
        off = offsetof(C64, flip);
        stride = sizeof(C64);
    } else {
        off = offsetof(C16, flip);
        stride = sizeof(C16);
    }
    CKB(b, cudaMemcpyAsync((unsigned char*)b->table + c * stride + off, &b->flip[c], sizeof(int32_t),
                           cudaMemcpyHostToDevice, b->stream));
    return CLB_OK;
}

extern "C" int clb_batch_init(clb_batch** out, int32_t ncase, const clb_params* p, const double* const* phi,
                              const clb_bc* bc, void* stream) {
    if (!out) return bfail(nullptr, CLB_ERR_ARG, "clb_batch_init: output pointer is NULL");
    *out = nullptr;
    if (ncase < 1 || !p || !phi || !bc) return bfail(nullptr, CLB_ERR_ARG, "clb_batch_init: bad arguments");
    for (int c = 1; c < ncase; ++c)
        if (p[c].precision != p[0].precision || p[c].shift != p[0].shift || p[c].forchheimer != p[0].forchheimer)
            return bfail(nullptr, CLB_ERR_ARG, "clb_batch_init: all cases must share precision, shift, forchheimer");
    clb_batch* b = new (std::nothrow) clb_batch();
    if (!b) return bfail(nullptr, CLB_ERR_OOM, "clb_batch_init: out of host memory");
    b->prec = p[0].precision;
    b->shift = p[0].shift;
    b->forch = p[0].forchheimer;
    b->stream = (cudaStream_t)stream;
    auto bail = [&](int code) {
        g_init_error = b->err.empty() ? g_init_error : b->err;
        clb_batch_destroy(b);
        return code;
    };
    for (int c = 0; c < ncase; ++c) {
        clb_handle* h = nullptr;
        const int rc = clb_init(&h, &p[c], phi[c], nullptr, &bc[c], stream);
        if (rc != CLB_OK) {
            bfail(b, rc, "clb_batch_init: case %d: %s", c, g_init_error.c_str());
            return bail(rc);
        }
        b->cases.push_back(h);
        b->active.push_back(1);
        b->flip.push_back(0);
    }
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        bfail(b, CLB_ERR_CUDA, "clb_batch_init: stream creation failed");
        return bail(CLB_ERR_CUDA);
    }
    // device table of the cases
    size_t bytes;
    std::vector<unsigned char> host;
    if (b->prec == CLB_F64) {
        std::vector<CaseT<double, double>> t(ncase);
        for (int c = 0; c < ncase; ++c) {
            clb_handle* h = b->cases[c];
            t[c].K = h->k64;
            t[c].A = h->aux64();
            t[c].b[0] = h->buf<double>(0);
            t[c].b[1] = h->buf<double>(1);
            t[c].flip = 0;
        }
        bytes = t.size() * sizeof(t[0]);
        host.assign((unsigned char*)t.data(), (unsigned char*)t.data() + bytes);
    } else {
        std::vector<CaseT<float, __half>> t(ncase);
        for (int c = 0; c < ncase; ++c) {
            clb_handle* h = b->cases[c];
            t[c].K = h->k32;
            t[c].A = h->aux32();
            t[c].b[0] = h->buf<__half>(0);
            t[c].b[1] = h->buf<__half>(1);
            t[c].flip = 0;
        }
        bytes = t.size() * sizeof(t[0]);
        host.assign((unsigned char*)t.data(), (unsigned char*)t.data() + bytes);
    }
    if (cudaMalloc(&b->table, bytes) != cudaSuccess ||
        cudaMemcpy(b->table, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        bfail(b, CLB_ERR_CUDA, "clb_batch_init: case table upload failed");
        return bail(CLB_ERR_CUDA);
    }
    if (cudaMalloc(&b->bar, sizeof(GridBarrier)) != cudaSuccess ||
        cudaMemset(b->bar, 0, sizeof(GridBarrier)) != cudaSuccess) {
        bfail(b, CLB_ERR_CUDA, "clb_batch_init: grid barrier allocation failed");
        return bail(CLB_ERR_CUDA);
    }
    const int rc = batch_build_tiles(b);
    if (rc != CLB_OK) return bail(rc);
    *out = b;
    return CLB_OK;
}

extern "C" int clb_batch_step(clb_batch* b, int64_t n) {
    if (!b) return CLB_ERR_ARG;
    if (n < 0) return bfail(b, CLB_ERR_ARG, "clb_batch_step: negative step count");
    int64_t left = n;
    while (left > 0) {
        if (left >= kGraphSteps && !b->graph_failed) {
            if (!b->graph[b->par]) {
                b->graph[b->par] = batch_capture(b, b->par);
                if (!b->graph[b->par]) {
                    b->graph_failed = true;
                    continue;
                }
            }
            CKB(b, cudaGraphLaunch(b->graph[b->par], b->stream));   // even count: parity unchanged
            left -= kGraphSteps;
        } else if (b->mode == CLB_BATCH_PERSISTENT) {
            const int k = (int)std::min<int64_t>(left, kGraphSteps);
            const cudaError_t e = batch_persist(b, b->stream, b->par, k, 0, b->wait_limit);
            if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
                // the device cannot hold the whole grid at once: step by launches instead
                cudaGetLastError();
                b->mode = CLB_BATCH_GRAPH;
                batch_drop_graphs(b);
                continue;
            }
            CKB(b, e);
            b->par ^= k & 1;
            left -= k;
        } else {
            batch_launch(b, b->stream);
            CKB(b, cudaGetLastError());
            left -= 1;
        }
    }
    b->t += n;
    batch_sync_cases(b);
    for (size_t c = 0; c < b->cases.size(); ++c)
        if (b->active[c]) b->cases[c]->t += n;
    return CLB_OK;
}

// Waits for the batch's stream and reports a grid barrier that gave up
// (persistent mode) as CLB_ERR_TIMEOUT, clearing the flag.
static int batch_check(clb_batch* b) {
    CKB(b, cudaStreamSynchronize(b->stream));
    if (!b->bar) return CLB_OK;
    unsigned failed = 0;
    CKB(b, cudaMemcpy(&failed, &b->bar->failed, sizeof failed, cudaMemcpyDeviceToHost));
    if (!failed) return CLB_OK;
    CKB(b, cudaMemset(&b->bar->failed, 0, sizeof failed));
    return bfail(b, CLB_ERR_TIMEOUT,
                 "persistent batch: a grid barrier wait expired; the state of the steps since the last check is "
                 "not valid");
}

extern "C" int clb_batch_set_mode(clb_batch* b, int32_t mode) {
    if (!b) return CLB_ERR_ARG;
    if (mode != CLB_BATCH_GRAPH && mode != CLB_BATCH_PERSISTENT)
        return bfail(b, CLB_ERR_ARG, "clb_batch_set_mode: mode must be CLB_BATCH_GRAPH or CLB_BATCH_PERSISTENT");
    const int rc = batch_check(b);
    if (rc != CLB_OK) return rc;
    b->mode = mode;
    batch_drop_graphs(b);
    return CLB_OK;
}

extern "C" int clb_batch_barrier_selftest(clb_batch* b, int64_t limit_cycles) {
    if (!b) return CLB_ERR_ARG;
    if (limit_cycles < 1 || limit_cycles > 4000000000LL)
        return bfail(b, CLB_ERR_ARG, "clb_batch_barrier_selftest: limit outside 1 .. 4e9 cycles");
    int rc = batch_check(b);
    if (rc != CLB_OK) return rc;
    // one step whose barrier waits for one block more than the launch has:
    // the wait must expire; the step wrote only the unused buffer, so the
    // state (parity, time) stays as it was
    CKB(b, batch_persist(b, b->stream, b->par, 1, 1, (long long)limit_cycles));
    return batch_check(b);
}

extern "C" int clb_batch_set_active(clb_batch* b, const int32_t* active) {
    if (!b || !active) return CLB_ERR_ARG;
    batch_sync_cases(b);
    for (size_t c = 0; c < b->cases.size(); ++c) {
        const int32_t now = active[c] != 0;
        if (now && !b->active[c]) {
            // resume from the buffer the case was retired in
            b->flip[c] = b->cases[c]->par ^ b->par;
            const int rc = batch_upload_flip(b, c);
            if (rc != CLB_OK) return rc;
        }
        b->active[c] = now;
    }
    return batch_build_tiles(b);
}

extern "C" int clb_batch_nusselt(clb_batch* b, int32_t side, double* nu) {
    if (!b || !nu) return CLB_ERR_ARG;
    const int rb = batch_check(b);
    if (rb != CLB_OK) return rb;
    batch_sync_cases(b);
    for (size_t c = 0; c < b->cases.size(); ++c) {
        const int rc = clb_nusselt(b->cases[c], side, &nu[c]);
        if (rc != CLB_OK) return bfail(b, rc, "clb_batch_nusselt: case %zu: %s", c, b->cases[c]->err.c_str());
    }
    return CLB_OK;
}

extern "C" int clb_batch_macros(clb_batch* b, int32_t c, double* rho, double* ux, double* uy, double* T) {
    if (!b || c < 0 || c >= (int32_t)b->cases.size()) return CLB_ERR_ARG;
    const int rb = batch_check(b);
    if (rb != CLB_OK) return rb;
    batch_sync_cases(b);
    const int rc = clb_macros(b->cases[c], rho, ux, uy, T);
    if (rc != CLB_OK) return bfail(b, rc, "clb_batch_macros: case %d: %s", c, b->cases[c]->err.c_str());
    return CLB_OK;
}

extern "C" int clb_batch_tune(clb_batch* b, int32_t steps, int32_t* chosen) {
    if (!b || steps < 1) return CLB_ERR_ARG;
    cudaEvent_t e0, e1;
    CKB(b, cudaEventCreate(&e0));
    CKB(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_s = b->shape, best_p = b->per_cta;
    for (int s = 0; s < kNumShapes; ++s)
        for (int q = 0; q < 3; ++q) {
            b->shape = s;
            b->per_cta = kPerCta[q];
            int rc = batch_build_tiles(b);
            if (rc != CLB_OK) return rc;
            batch_launch(b, b->stream);   // warm-up step of this shape
            CKB(b, cudaEventRecord(e0, b->stream));
            for (int i = 0; i < steps; ++i) batch_launch(b, b->stream);
            CKB(b, cudaEventRecord(e1, b->stream));
            CKB(b, cudaEventSynchronize(e1));
            CKB(b, cudaGetLastError());
            float ms = 0.0f;
            CKB(b, cudaEventElapsedTime(&ms, e0, e1));
            b->t += steps + 1;
            for (size_t c = 0; c < b->cases.size(); ++c)
                if (b->active[c]) b->cases[c]->t += steps + 1;
            if (ms < best) {
                best = ms;
                best_s = s;
                best_p = kPerCta[q];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->shape = best_s;
    b->per_cta = best_p;
    batch_sync_cases(b);
    if (chosen) *chosen = best_s * 3 + (best_p == kPerCta[0] ? 0 : best_p == kPerCta[1] ? 1 : 2);
    return batch_build_tiles(b);
}

extern "C" int clb_batch_set_tiling(clb_batch* b, int32_t choice) {
    if (!b) return CLB_ERR_ARG;
    if (choice < 0 || choice >= kNumShapes * 3)
        return bfail(b, CLB_ERR_ARG, "clb_batch_set_tiling: choice %d outside [0, %d)", choice, kNumShapes * 3);
    b->shape = choice / 3;
    b->per_cta = kPerCta[choice % 3];
    return batch_build_tiles(b);
}

extern "C" int64_t clb_batch_nodes(const clb_batch* b) { return b ? b->nodes : -1; }

extern "C" int64_t clb_batch_time(const clb_batch* b) { return b ? b->t : -1; }

extern "C" int clb_batch_sync(clb_batch* b) {
    if (!b) return CLB_ERR_ARG;
    return batch_check(b);
}

extern "C" const char* clb_batch_last_error(const clb_batch* b) { return b ? b->err.c_str() : g_init_error.c_str(); }

extern "C" void clb_batch_destroy(clb_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (clb_handle* h : b->cases) clb_destroy(h);
    cudaFree(b->bar);
    cudaFree(b->table);
    cudaFree(b->tiles);
    cudaFree(b->itiles);
    cudaFree(b->echunks);
    cudaFree(b->work);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->cap_side) cudaStreamDestroy(b->cap_side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
}
