// blink_api.cu -- the C ABI declared in include/blink.h.
//
// Host-side runtime: argument validation, channel deduplication, device
// workspace (a per-context stream-ordered memory pool), per-size grouping of
// layers and kernel dispatch.  No compute happens on the host.
#include "blink.h"
#include "blink_common.cuh"
#include "blink_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

using blink::ChanGeom;
using blink::ChanInfo;
using blink::DevLayer;
using blink::Error;

struct blink_ctx {
    int device = 0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t copy_in = nullptr;   // host-buffer pipeline: host -> device copies
    cudaStream_t copy_out = nullptr;  // host-buffer pipeline: device -> host copies
    int64_t wait_ns = -1;             // bounded-wait limit of the tensor-core kernels (< 0: default)
    void *h_stage = nullptr;          // pinned staging of plan tables (host -> device copies)
    size_t h_stage_bytes = 0;
    cudaStream_t aux = nullptr;       // second stream of the large-image path
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
};

namespace {

// Pinned host buffer of at least `bytes` owned by the context, for the plan
// tables' copies: from pinned memory they are asynchronous DMA, where a
// pageable source makes the host wait for the stream to reach the copy.  The
// contents are not kept across calls; a context is used by one host thread
// and every plan build waits for its copies before it returns.
void *ctx_stage(blink_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->h_stage_bytes) return ctx->h_stage;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    const size_t want = std::max<size_t>(bytes, size_t(1) << 20);
    if (cudaHostAlloc(&ctx->h_stage, want, cudaHostAllocDefault) != cudaSuccess) {
        ctx->h_stage = nullptr;
        return nullptr;
    }
    ctx->h_stage_bytes = want;
    return ctx->h_stage;
}

}  // namespace

struct blink_plan {
    blink_ctx *ctx = nullptr;
    int n_ant = 0;
    int64_t nb = 0;
    int n_layers = 0;
    int n_chan = 0;
    bool any_uniform = false;
    std::vector<ChanGeom> geoms;
    std::vector<ChanInfo> infos;
    std::vector<int32_t> layer_chan;
    std::vector<int64_t> layer_out;  // out_offset per layer in group order
    struct Group {
        int n_px;
        int first;
        int count;
        int r_alloc;
        int sched_ok;   // every channel of the group has a gridding schedule
        int max_chunk;  // largest staging chunk among those channels
        int max_seg;    // longest per-chunk schedule segment among them
        int force_path = 0;       // autotuned kernel choice (0 = default)
        size_t wave_budget = 0;   // autotuned wave size of the two-kernel path
        int kmax = 0;             // max |k_u| over the group's channels
        int row_entries = 0;      // max kept baselines per support row over the group's channels
        int64_t cg_stride = 0;    // compact grid per layer (complex elements), 0 if not used
    };
    std::vector<Group> groups;
    // device memory (one pool allocation for the tables, one for scratch)
    char *d_block = nullptr;
    ChanGeom *d_geom = nullptr;
    ChanInfo *d_info = nullptr;
    uint32_t *d_codes = nullptr;
    float *d_wgt = nullptr;
    DevLayer *d_layers = nullptr;
    int2 *d_cells = nullptr;
    float2 *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    unsigned char *d_sched = nullptr;
    unsigned char *d_csr = nullptr;  // row buckets per channel
    size_t csr_bytes = 0;
    float2 *d_dscratch = nullptr;  // adjoint column-transform scratch (allocated on first use)
    size_t dscratch_bytes = 0;
    float2 *d_gscratch = nullptr;  // tensor-core transform scratch (allocated on first use)
    size_t gscratch_bytes = 0;
    int *d_status = nullptr;       // device status word (in the table block)
    int64_t out_extent = 0;        // max over layers of out_offset + n_px^2
    int *d_queue = nullptr;        // work queue of the persistent large-image kernel
    size_t queue_bytes = 0;
    float2 *d_cg = nullptr;        // compact grids of a wave of large-image layers
    size_t cg_bytes = 0;
    float2 *d_gprod = nullptr;     // gain-product table of the fused epilogue (on first use)
    size_t gprod_bytes = 0;
    double *d_sqpart = nullptr;    // per-layer partial sums of squares (on first use)
    float *d_imgtmp = nullptr;     // images of sizes without the fused adjoint columns when the
                                   // caller stores none (on first use; output extent)
    int sq_stride = 0;             // slots per layer: the most column items of any group
    cudaStream_t last_stream = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    cudaGraphExec_t graph = nullptr;     // captured image launches (blink_plan_capture)
};

namespace {

constexpr size_t kScratchCap = size_t(48) << 20;
// Compact grids of large-image layers per plan: one wave of the large path.
constexpr size_t kCgCap = size_t(128) << 20;
// Tensor-core transform scratch per plan: its waves trade L2 residency of the
// pass-1 output for fewer, fuller launches (each wave is three kernels).
constexpr size_t kTensorScratchCap = size_t(512) << 20;
// Largest gain-product table (distinct gain rows x baselines x 8 bytes) the
// fused epilogue builds; above it the kernels form g_i conj(g_j) per entry.
constexpr size_t kGainTableCap = size_t(256) << 20;  // bytes of row-transform scratch per plan (L2-sized waves)

// Runs f with ctx->device current and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(blink_ctx *ctx, int status, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return status;
}

int fail(blink_ctx *ctx, const Error &e) { return fail(ctx, e.status, e.msg); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct ChanKey {
    int32_t n_px, weighting;
    uint64_t freq_bits, du_bits;
    bool operator==(const ChanKey &o) const {
        return n_px == o.n_px && weighting == o.weighting && freq_bits == o.freq_bits &&
               du_bits == o.du_bits;
    }
};
struct ChanKeyHash {
    size_t operator()(const ChanKey &k) const {
        uint64_t h = k.freq_bits * 0x9E3779B97F4A7C15ull;
        h ^= (k.du_bits + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2));
        h ^= uint64_t(uint32_t(k.n_px)) * 0xC2B2AE3D27D4EB4Full + uint64_t(k.weighting);
        return size_t(h ^ (h >> 29));
    }
};

ChanKey key_of(const blink_layer &L) {
    ChanKey k;
    k.n_px = L.n_px;
    k.weighting = L.weighting;
    std::memcpy(&k.freq_bits, &L.freq_hz, 8);
    std::memcpy(&k.du_bits, &L.delta_u, 8);
    return k;
}

int validate(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
             int n_layers) {
    if (!ctx) return BLINK_ERR_INVALID;
    if (n_ant < 2) return fail(ctx, BLINK_ERR_INVALID, "n_ant must be >= 2");
    if (int64_t(n_ant) * (n_ant - 1) / 2 > (int64_t(1) << 31))
        return fail(ctx, BLINK_ERR_UNSUPPORTED, "too many baselines (n_ant too large)");
    if (!d_ant_xyz) return fail(ctx, BLINK_ERR_INVALID, "d_ant_xyz is NULL");
    if (n_layers < 0) return fail(ctx, BLINK_ERR_INVALID, "n_layers < 0");
    if (n_layers > 0 && !h_layers) return fail(ctx, BLINK_ERR_INVALID, "h_layers is NULL");
    for (int l = 0; l < n_layers; ++l) {
        const blink_layer &L = h_layers[l];
        const std::string at = " (layer " + std::to_string(l) + ")";
        if (L.n_px < 4 || (L.n_px & 1))
            return fail(ctx, BLINK_ERR_INVALID, "n_px must be even and >= 4" + at);
        if (!blink::image_size_supported(L.n_px))
            return fail(ctx, BLINK_ERR_UNSUPPORTED,
                        "image size " + std::to_string(L.n_px) + " not supported" + at);
        if (L.weighting != BLINK_NATURAL && L.weighting != BLINK_UNIFORM)
            return fail(ctx, BLINK_ERR_INVALID, "weighting must be 0 or 1" + at);
        if (!(std::isfinite(L.freq_hz) && L.freq_hz > 0))
            return fail(ctx, BLINK_ERR_INVALID, "freq_hz must be finite and > 0" + at);
        if (!(std::isfinite(L.delta_u) && L.delta_u > 0))
            return fail(ctx, BLINK_ERR_INVALID, "delta_u must be finite and > 0" + at);
        if (L.vis_offset < 0 || L.out_offset < 0)
            return fail(ctx, BLINK_ERR_INVALID, "offsets must be >= 0" + at);
    }
    return BLINK_OK;
}

void free_plan_memory(blink_plan *p, cudaStream_t st) {
    if (p->d_block) cudaFreeAsync(p->d_block, st);
    if (p->d_scratch) cudaFreeAsync(p->d_scratch, st);
    if (p->d_sched) cudaFreeAsync(p->d_sched, st);
    if (p->d_csr) cudaFreeAsync(p->d_csr, st);
    p->d_csr = nullptr;
    p->csr_bytes = 0;
    if (p->d_dscratch) cudaFreeAsync(p->d_dscratch, st);
    if (p->d_gscratch) cudaFreeAsync(p->d_gscratch, st);
    p->d_gscratch = nullptr;
    if (p->d_gprod) cudaFreeAsync(p->d_gprod, st);
    p->d_gprod = nullptr;
    if (p->d_sqpart) cudaFreeAsync(p->d_sqpart, st);
    p->d_sqpart = nullptr;
    if (p->d_imgtmp) cudaFreeAsync(p->d_imgtmp, st);
    p->d_imgtmp = nullptr;
    if (p->d_queue) cudaFreeAsync(p->d_queue, st);
    p->d_queue = nullptr;
    p->queue_bytes = 0;
    if (p->d_cg) cudaFreeAsync(p->d_cg, st);
    p->d_cg = nullptr;
    p->cg_bytes = 0;
    p->gprod_bytes = 0;
    p->d_block = nullptr;
    p->d_scratch = nullptr;
    p->d_sched = nullptr;
    p->d_dscratch = nullptr;
}

// Images up to this size are gridded by the fused kernels, which can use the
// register-accumulation schedule.
constexpr int kSchedMaxPx = 256;
// Plan tables above this many bytes are copied from the context's pinned buffer.
constexpr size_t kPinnedStageMin = 64 * 1024;

// Builds the channel tables of a plan on `st` and waits for them.
int build_plan(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
               int n_layers, bool want_cells, blink_plan *p, cudaStream_t st) {
    p->ctx = ctx;
    p->n_ant = n_ant;
    p->nb = int64_t(n_ant) * (n_ant - 1) / 2;
    for (int l = 0; l < n_layers; ++l)
        p->out_extent = std::max(p->out_extent, h_layers[l].out_offset + int64_t(h_layers[l].n_px) * h_layers[l].n_px);
    p->n_layers = n_layers;
    p->last_stream = st;
    // distinct channels
    std::unordered_map<ChanKey, int, ChanKeyHash> chan_of;
    chan_of.reserve(64);
    p->layer_chan.resize(size_t(n_layers));
    int prev_chan = -1;
    ChanKey prev_key{};
    for (int l = 0; l < n_layers; ++l) {
        const ChanKey k = key_of(h_layers[l]);
        int c;
        if (prev_chan >= 0 && k == prev_key) {
            c = prev_chan;
        } else {
            auto it = chan_of.find(k);
            if (it == chan_of.end()) {
                c = int(p->geoms.size());
                chan_of.emplace(k, c);
                p->geoms.push_back(ChanGeom{h_layers[l].freq_hz, h_layers[l].delta_u,
                                            h_layers[l].n_px, h_layers[l].weighting});
            } else {
                c = it->second;
            }
        }
        p->layer_chan[size_t(l)] = c;
        prev_chan = c;
        prev_key = k;
    }
    p->n_chan = int(p->geoms.size());
    // the array's extent, for the compact-support bound of large sizes
    double span_x = -1.0, span_y = -1.0;
    bool any_large = false;
    for (const auto &g : p->geoms) any_large = any_large || g.n_px > kSchedMaxPx;
    if (any_large && n_ant > 0) {
        std::vector<double> hx(size_t(3) * size_t(n_ant));
        if (cudaMemcpyAsync(hx.data(), d_ant_xyz, sizeof(double) * hx.size(), cudaMemcpyDeviceToHost, st) ==
                cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess) {
            double x0 = hx[0], x1 = hx[0], y0 = hx[1], y1 = hx[1];
            for (int a = 1; a < n_ant; ++a) {
                x0 = std::min(x0, hx[3 * a]);
                x1 = std::max(x1, hx[3 * a]);
                y0 = std::min(y0, hx[3 * a + 1]);
                y1 = std::max(y1, hx[3 * a + 1]);
            }
            span_x = x1 - x0;
            span_y = y1 - y0;
        }
    }
    // channel table offsets
    p->infos.assign(size_t(p->n_chan), ChanInfo{});
    int64_t wgt_total = 0;
    int64_t sched_total = 0;
    int64_t csr_total = 0;
    for (int c = 0; c < p->n_chan; ++c) {
        ChanInfo &ci = p->infos[size_t(c)];
        ci.n_px = p->geoms[size_t(c)].n_px;
        ci.weighting = p->geoms[size_t(c)].weighting;
        ci.code_off = int64_t(c) * p->nb;
        ci.sched_off = -1;
        // row buckets only where a full-extent image can miss the fused kernel
        // (sizes whose whole support always fits it never need them)
        if (!blink::image_small_path(ci.n_px, ci.n_px / 2 + 1)) {
            ci.csr_off = csr_total;
            csr_total += blink::CsrLayout(ci.n_px, p->nb).bytes;
        } else {
            ci.csr_off = -1;
        }
        // register-accumulation schedule: sizes <= 256 (the fused kernel), and
        // larger sizes whose compact support is sure to fit (the compact
        // gridding kernel)
        const bool sched_large = ci.n_px > kSchedMaxPx && span_x >= 0.0 &&
                                 blink::cg_bound_fits(span_x, span_y, p->geoms[size_t(c)].freq_hz,
                                                      p->geoms[size_t(c)].delta_u, ci.n_px);
        const bool sched = ci.n_px <= kSchedMaxPx || sched_large;
        ci.sched_large = sched_large ? 1 : 0;
        if (sched) {
            const int q = int((p->nb + blink::kSchedMaxChunk - 1) / blink::kSchedMaxChunk);
            int k = int((p->nb + q - 1) / q);
            k += k & 1;
            ci.n_chunks = q;
            ci.chunk = k;
            ci.sched_off = sched_total;
            sched_total += blink::SchedLayout(ci.n_px, p->nb, q).bytes;
        }
        if (ci.weighting == BLINK_UNIFORM || sched) {
            ci.wgt_off = wgt_total;
            wgt_total += int64_t(ci.n_px / 2) * ci.n_px;
            p->any_uniform = true;
        } else {
            ci.wgt_off = -1;
        }
    }
    // layers grouped by image size, stable within a size
    std::vector<int> order(static_cast<size_t>(n_layers));
    for (int l = 0; l < n_layers; ++l) order[size_t(l)] = l;
    bool grouped = true;
    for (int l = 1; l < n_layers && grouped; ++l) grouped = h_layers[l - 1].n_px <= h_layers[l].n_px;
    if (!grouped)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return h_layers[a].n_px < h_layers[b].n_px; });
    // geometry, channel and layer tables: large ones staged in the context's
    // pinned buffer (asynchronous DMA), small ones copied from pageable memory,
    // which the driver passes inline with less latency than a DMA
    const size_t sz_geom = align_up(sizeof(ChanGeom) * size_t(p->n_chan), 256);
    const size_t sz_info = align_up(sizeof(ChanInfo) * size_t(p->n_chan), 256);
    const size_t sz_all = sz_geom + sz_info + sizeof(DevLayer) * size_t(std::max(n_layers, 1));
    std::vector<char> h_small;
    char *hs = nullptr;
    if (sz_all > kPinnedStageMin) {
        hs = static_cast<char *>(ctx_stage(ctx, sz_all));
        if (!hs) return fail(ctx, BLINK_ERR_WORKSPACE, "pinned staging allocation failed");
    } else {
        h_small.resize(sz_all);
        hs = h_small.data();
    }
    ChanGeom *h_geom = reinterpret_cast<ChanGeom *>(hs);
    ChanInfo *h_info = reinterpret_cast<ChanInfo *>(hs + sz_geom);
    DevLayer *dl = reinterpret_cast<DevLayer *>(hs + sz_geom + sz_info);
    for (int k = 0; k < n_layers; ++k) {
        const int l = order[size_t(k)];
        dl[size_t(k)] = DevLayer{h_layers[l].vis_offset, h_layers[l].out_offset,
                                 p->layer_chan[size_t(l)], l};
        p->layer_out.push_back(h_layers[l].out_offset);
        if (p->groups.empty() || p->groups.back().n_px != h_layers[l].n_px)
            p->groups.push_back(blink_plan::Group{h_layers[l].n_px, k, 0, 1, 0, 0, 0, 0, 0});
        p->groups.back().count++;
    }
    // one device block for every table
    const size_t a = 256;
    size_t off = 0;
    const size_t o_geom = off; off = align_up(off + sizeof(ChanGeom) * size_t(p->n_chan), a);
    const size_t o_info = off; off = align_up(off + sizeof(ChanInfo) * size_t(p->n_chan), a);
    const size_t o_codes = off; off = align_up(off + sizeof(uint32_t) * size_t(p->n_chan) * size_t(p->nb), a);
    const size_t o_wgt = off; off = align_up(off + sizeof(float) * size_t(std::max<int64_t>(wgt_total, 1)), a);
    const size_t o_layers = off; off = align_up(off + sizeof(DevLayer) * size_t(std::max(n_layers, 1)), a);
    const size_t o_status = off; off = align_up(off + sizeof(int), a);
    const size_t o_cells = off;
    if (want_cells) off = align_up(off + sizeof(int2) * size_t(p->n_chan) * size_t(p->nb), a);
    void *blk = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&blk, std::max<size_t>(off, a), ctx->pool, st);
    if (e != cudaSuccess)
        return fail(ctx, BLINK_ERR_WORKSPACE, std::string("table allocation: ") + cudaGetErrorString(e));
    p->d_block = static_cast<char *>(blk);
    p->d_geom = reinterpret_cast<ChanGeom *>(p->d_block + o_geom);
    p->d_info = reinterpret_cast<ChanInfo *>(p->d_block + o_info);
    p->d_codes = reinterpret_cast<uint32_t *>(p->d_block + o_codes);
    p->d_wgt = reinterpret_cast<float *>(p->d_block + o_wgt);
    p->d_layers = reinterpret_cast<DevLayer *>(p->d_block + o_layers);
    p->d_cells = want_cells ? reinterpret_cast<int2 *>(p->d_block + o_cells) : nullptr;
    p->d_status = reinterpret_cast<int *>(p->d_block + o_status);
#define TRY(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, BLINK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    if (p->n_chan) {
        std::copy(p->geoms.begin(), p->geoms.end(), h_geom);
        std::copy(p->infos.begin(), p->infos.end(), h_info);
        TRY(cudaMemcpyAsync(p->d_geom, h_geom, sizeof(ChanGeom) * p->geoms.size(), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(p->d_info, h_info, sizeof(ChanInfo) * p->infos.size(), cudaMemcpyHostToDevice, st));
    }
    if (n_layers)
        TRY(cudaMemcpyAsync(p->d_layers, dl, sizeof(DevLayer) * size_t(n_layers), cudaMemcpyHostToDevice, st));
    if (p->any_uniform) TRY(cudaMemsetAsync(p->d_wgt, 0, sizeof(float) * size_t(wgt_total), st));
    TRY(cudaMemsetAsync(p->d_status, 0, sizeof(int), st));
    if (sched_total) {
        void *sb = nullptr;
        e = cudaMallocFromPoolAsync(&sb, size_t(sched_total), ctx->pool, st);
        if (e != cudaSuccess)
            return fail(ctx, BLINK_ERR_WORKSPACE, std::string("schedule allocation: ") + cudaGetErrorString(e));
        p->d_sched = static_cast<unsigned char *>(sb);
        TRY(cudaMemsetAsync(p->d_sched, 0, size_t(sched_total), st));
    }
    if (csr_total) {
        void *cb = nullptr;
        e = cudaMallocFromPoolAsync(&cb, size_t(csr_total), ctx->pool, st);
        if (e != cudaSuccess)
            return fail(ctx, BLINK_ERR_WORKSPACE, std::string("row-bucket allocation: ") + cudaGetErrorString(e));
        p->d_csr = static_cast<unsigned char *>(cb);
        p->csr_bytes = size_t(csr_total);
        TRY(cudaMemsetAsync(p->d_csr, 0, size_t(csr_total), st));
    }
    Error er = blink::launch_tables(d_ant_xyz, n_ant, p->nb, p->n_chan, p->d_geom, p->d_info,
                                    p->d_codes, p->d_cells, p->d_wgt, p->any_uniform, st, p->d_sched,
                                    p->d_csr);
    if (er.status) return fail(ctx, er);
    if (p->n_chan)
        TRY(cudaMemcpyAsync(h_info, p->d_info, sizeof(ChanInfo) * p->infos.size(), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    std::copy(h_info, h_info + p->infos.size(), p->infos.begin());
    // support rows per size group, scratch for the large-image path
    size_t scratch = 0, cg_need = 0;
    for (auto &g : p->groups) {
        int r = 1;
        g.sched_ok = p->d_sched != nullptr;
        g.max_chunk = 0;
        g.max_seg = 0;
        for (int k = g.first; k < g.first + g.count; ++k) {
            const ChanInfo &ci = p->infos[size_t(dl[size_t(k)].chan)];
            r = std::max(r, ci.rows);
            g.sched_ok = g.sched_ok && ci.sched_off >= 0 && ci.sched == 1;
            g.max_chunk = std::max(g.max_chunk, ci.chunk);
            g.max_seg = std::max(g.max_seg, ci.max_seg);
            g.kmax = std::max(g.kmax, ci.kmax_u);
            g.row_entries = std::max(g.row_entries, int(ci.n_kept / std::max(1, ci.rows)));
        }
        g.r_alloc = r;
        const size_t per = blink::image_scratch_per_layer(g.n_px, r);
        if (per) scratch = std::max(scratch, std::max(per, std::min(per * size_t(g.count), kScratchCap)));
        // compact gridding: every channel has its sorted chunk tables and the
        // group's largest compact grid fits the kernel's shared memory
        bool cg_ok = p->d_csr != nullptr && blink::cg_fits(r, g.kmax);
        for (int k = g.first; k < g.first + g.count && cg_ok; ++k)
            cg_ok = p->infos[size_t(dl[size_t(k)].chan)].csr_off >= 0;
        g.cg_stride = cg_ok ? (blink::cg_cells(r, g.kmax) + 1) & ~int64_t(1) : 0;
        if (cg_ok)
            cg_need = std::max(cg_need, std::min(size_t(g.count), std::max<size_t>(1, kCgCap / size_t(8 * g.cg_stride))) *
                                            size_t(8 * g.cg_stride));
    }
    // work queue of the persistent large-image kernel: sized for the largest
    // group, so every group (also one forced onto that path) can use it
    {
        size_t qb = 0;
        for (const auto &g : p->groups) qb = std::max(qb, blink::image_queue_bytes(g.count));
        void *q = nullptr;
        e = cudaMallocFromPoolAsync(&q, qb, ctx->pool, st);
        if (e != cudaSuccess)
            return fail(ctx, BLINK_ERR_WORKSPACE, std::string("work-queue allocation: ") + cudaGetErrorString(e));
        p->d_queue = static_cast<int *>(q);
        p->queue_bytes = qb;
    }
    if (cg_need) {
        void *c = nullptr;
        e = cudaMallocFromPoolAsync(&c, cg_need, ctx->pool, st);
        if (e != cudaSuccess)
            return fail(ctx, BLINK_ERR_WORKSPACE, std::string("compact-grid allocation: ") + cudaGetErrorString(e));
        p->d_cg = static_cast<float2 *>(c);
        p->cg_bytes = cg_need;
    }
    if (scratch) {
        void *s = nullptr;
        e = cudaMallocFromPoolAsync(&s, scratch, ctx->pool, st);
        if (e != cudaSuccess)
            return fail(ctx, BLINK_ERR_WORKSPACE, std::string("scratch allocation: ") + cudaGetErrorString(e));
        p->d_scratch = static_cast<float2 *>(s);
        p->scratch_bytes = scratch;
    }
#undef TRY
    return BLINK_OK;
}

// Complex elements of the kept adjoint columns before group g (slots of
// r_alloc rows of N per layer, groups in plan order); g == groups: the total.
static int64_t adjoint_offset(const blink_plan *p, size_t g) {
    int64_t off = 0;
    for (size_t k = 0; k < g && k < p->groups.size(); ++k)
        off += int64_t(p->groups[k].count) * p->groups[k].r_alloc * p->groups[k].n_px;
    return off;
}

blink::ImageArgs group_args(const blink_plan *p, const blink_plan::Group &g, const float *d_vis,
                            void *out, float *d_wsum, uint32_t flags) {
    blink::ImageArgs a{};
    a.vis = reinterpret_cast<const float2 *>(d_vis);
    a.out = out;
    a.wsum_out = d_wsum;
    a.layers = p->d_layers + g.first;
    a.n_layers = g.count;
    a.chans = p->d_info;
    a.codes = p->d_codes;
    a.wgt = p->d_wgt;
    a.nb = p->nb;
    a.flags = flags;
    a.r_alloc = g.r_alloc;
    a.scratch = p->d_scratch;
    a.scratch_bytes = p->scratch_bytes;
    a.sched = p->d_sched;
    a.sched_ok = g.sched_ok;
    a.max_chunk = g.max_chunk;
    a.max_seg = g.max_seg;
    a.status = p->d_status;
    a.csr = p->d_csr;
    a.n_ant = p->n_ant;
    a.wait_ns = p->ctx->wait_ns;
    a.kmax = g.kmax;
    a.force_path = g.force_path;
    a.wave_budget = g.wave_budget;
    a.aux = p->ctx->aux;
    a.ev_fork = p->ctx->ev_fork;
    a.ev_join = p->ctx->ev_join;
    a.queue = p->d_queue;
    a.queue_bytes = p->queue_bytes;
    a.csr_bytes = p->csr_bytes;
    a.row_entries = g.row_entries;
    if (g.cg_stride > 0 && p->d_cg) {
        a.cg = p->d_cg;
        a.cg_stride = g.cg_stride;
        a.cg_cap = int(std::min<size_t>(size_t(g.count), p->cg_bytes / size_t(8 * g.cg_stride)));
    }
    return a;
}

}  // namespace

extern "C" {

int blink_abi_version(void) { return BLINK_ABI_VERSION; }

int blink_supported_sizes(int32_t *sizes, int cap) { return blink::supported_sizes(sizes, cap); }

int blink_ctx_create(blink_ctx **out, int device) {
    if (!out) return BLINK_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return BLINK_ERR_INVALID;
    blink_ctx *ctx = new (std::nothrow) blink_ctx();
    if (!ctx) return BLINK_ERR_WORKSPACE;
    ctx->device = device;
    DeviceGuard g(device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) {
        delete ctx;
        return BLINK_ERR_CUDA;
    }
    uint64_t keep = std::numeric_limits<uint64_t>::max();
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        blink_ctx_destroy(ctx);
        return BLINK_ERR_CUDA;
    }
    *out = ctx;
    return BLINK_OK;
}

void blink_ctx_destroy(blink_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
        if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
        if (ctx->aux) cudaStreamDestroy(ctx->aux);
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    }
    delete ctx;
}

const char *blink_last_error(const blink_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int blink_plan_create(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
                      int n_layers, blink_plan **out, void *stream) {
    if (!ctx || !out) return BLINK_ERR_INVALID;
    *out = nullptr;
    int st = validate(ctx, d_ant_xyz, n_ant, h_layers, n_layers);
    if (st) return st;
    DeviceGuard g(ctx->device);
    blink_plan *p = new (std::nothrow) blink_plan();
    if (!p) return fail(ctx, BLINK_ERR_WORKSPACE, "host allocation failed");
    st = build_plan(ctx, d_ant_xyz, n_ant, h_layers, n_layers, false, p, static_cast<cudaStream_t>(stream));
    if (st) {
        free_plan_memory(p, static_cast<cudaStream_t>(stream));
        delete p;
        return st;
    }
    ctx->err.clear();
    *out = p;
    return BLINK_OK;
}

// Row-transform scratch for every group that may take the two-kernel path
// (needed before autotuning or graph capture, which must not allocate).
static int ensure_rows_scratch(blink_plan *p, cudaStream_t st) {
    size_t need = 0;
    for (const auto &grp : p->groups) {
        const size_t per = blink::image_rows_scratch_per_layer(grp.n_px, grp.r_alloc);
        need = std::max(need, std::max(per, std::min(per * size_t(grp.count), kScratchCap)));
    }
    if (need <= p->scratch_bytes) return BLINK_OK;
    if (p->d_scratch) cudaFreeAsync(p->d_scratch, st);
    p->d_scratch = nullptr;
    p->scratch_bytes = 0;
    void *ptr = nullptr;
    const cudaError_t e = cudaMallocFromPoolAsync(&ptr, need, p->ctx->pool, st);
    if (e != cudaSuccess) return fail(p->ctx, BLINK_ERR_WORKSPACE, "scratch allocation failed");
    p->d_scratch = static_cast<float2 *>(ptr);
    p->scratch_bytes = need;
    return BLINK_OK;
}

int blink_plan_image(blink_plan *p, const float *d_vis, float *d_images, float *d_wsum, uint32_t flags,
                     void *stream) {
    return blink_plan_image_ex(p, d_vis, d_images, d_wsum, flags, nullptr, stream);
}

int blink_plan_image_ex(blink_plan *p, const float *d_vis, float *d_images, float *d_wsum, uint32_t flags,
                        const blink_epilogue *epi, void *stream) {
    if (!p) return BLINK_ERR_INVALID;
    blink_ctx *ctx = p->ctx;
    if (p->n_layers && (!d_vis || (!d_images && !(epi && epi->d_adjoint))))
        return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    const uint32_t mode = (flags & BLINK_TRANSFORM_MASK) >> 4;
    if ((flags & ~uint32_t(BLINK_NORMALIZE | BLINK_TRANSFORM_MASK)) || mode > 4)
        return fail(ctx, BLINK_ERR_INVALID, "unknown flags");
    const float *d_gains = epi ? epi->d_gains : nullptr;
    const float *d_ref = epi ? epi->d_ref : nullptr;
    double *d_sqnorm = epi ? epi->d_sqnorm : nullptr;
    float *d_adjoint = epi ? epi->d_adjoint : nullptr;
    if (d_adjoint && (reinterpret_cast<uintptr_t>(d_adjoint) & 7))
        return fail(ctx, BLINK_ERR_INVALID, "adjoint buffer must be 8-byte aligned");
    if (epi && (epi->gain_stride < 0 || epi->gain_period < 0))
        return fail(ctx, BLINK_ERR_INVALID, "gain_stride and gain_period must be >= 0");
    if (d_gains && p->n_ant >= 65536) return fail(ctx, BLINK_ERR_UNSUPPORTED, "gains need fewer than 65536 antennas");
    if (d_ref && d_images) {
        // the kernels read the reference and write the output through
        // non-aliasing (restrict) pointers: the two extents must not overlap
        const uintptr_t r0 = reinterpret_cast<uintptr_t>(d_ref), i0 = reinterpret_cast<uintptr_t>(d_images);
        const uintptr_t ext = uintptr_t(p->out_extent) * sizeof(float);
        if (r0 < i0 + ext && i0 < r0 + ext)
            return fail(ctx, BLINK_ERR_INVALID, "reference images overlap the output");
    }
    if (d_sqnorm && mode)
        return fail(ctx, BLINK_ERR_UNSUPPORTED, "per-layer sums of squares need the FFT transform (no tensor-core mode)");
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    p->last_stream = st;
    if (d_sqnorm && !p->d_sqpart && p->n_layers) {
        int stride = 1;
        for (const auto &grp : p->groups) stride = std::max(stride, blink::sq_slots(grp.n_px));
        void *ptr = nullptr;
        const cudaError_t e =
            cudaMallocFromPoolAsync(&ptr, size_t(p->n_layers) * size_t(stride) * sizeof(double), ctx->pool, st);
        if (e != cudaSuccess)
            return fail(ctx, BLINK_ERR_WORKSPACE, std::string("partial sums of squares: ") + cudaGetErrorString(e));
        p->d_sqpart = static_cast<double *>(ptr);
        p->sq_stride = stride;
    }
    // gain products g_i conj(g_j) once per distinct gain row, when they fit
    const float2 *gprod = nullptr;
    if (d_gains && p->nb > 0) {
        const int64_t rows = epi->gain_stride == 0 ? 1
                             : (epi->gain_period > 0 ? std::min<int64_t>(epi->gain_period, p->n_layers)
                                                     : int64_t(p->n_layers));
        const size_t bytes = size_t(rows) * size_t(p->nb) * sizeof(float2);
        if (rows > 0 && bytes <= kGainTableCap) {
            if (bytes > p->gprod_bytes) {
                if (p->d_gprod) cudaFreeAsync(p->d_gprod, st);
                p->d_gprod = nullptr;
                p->gprod_bytes = 0;
                void *ptr = nullptr;
                if (cudaMallocFromPoolAsync(&ptr, bytes, ctx->pool, st) != cudaSuccess)
                    return fail(ctx, BLINK_ERR_WORKSPACE, "gain-product table allocation failed");
                p->d_gprod = static_cast<float2 *>(ptr);
                p->gprod_bytes = bytes;
            }
            Error e = blink::launch_gain_products(reinterpret_cast<const float2 *>(d_gains), epi->gain_stride,
                                                  int(rows), p->n_ant, p->nb, p->d_gprod, st);
            if (e.status) return fail(ctx, e);
            gprod = p->d_gprod;
        }
    }
    // groups that take the tensor-core transform: supported size, 16-byte
    // aligned image rows (and reference rows)
    auto gemm_ok = [&](const blink_plan::Group &grp) {
        if (!mode || !blink::dftgemm_supported(grp.n_px, grp.r_alloc, mode) ||
            ((reinterpret_cast<uintptr_t>(d_images) | reinterpret_cast<uintptr_t>(d_ref)) & 15))
            return false;
        for (int k = grp.first; k < grp.first + grp.count; ++k)
            if (p->layer_out[size_t(k)] & 3) return false;
        return true;
    };
    if (mode && !p->d_gscratch) {
        size_t need = 0;
        for (const auto &grp : p->groups) {
            if (!gemm_ok(grp)) continue;
            const size_t per = blink::dftgemm_scratch_per_layer(grp.n_px, grp.r_alloc);
            const size_t fixed = blink::dftgemm_scratch_fixed(grp.n_px, grp.r_alloc, grp.kmax);
            need = std::max(need, fixed + std::max(per, std::min(per * size_t(grp.count), kTensorScratchCap)));
        }
        if (need) {
            void *ptr = nullptr;
            const cudaError_t e = cudaMallocFromPoolAsync(&ptr, need, ctx->pool, st);
            if (e != cudaSuccess)
                return fail(ctx, BLINK_ERR_WORKSPACE, std::string("tensor-core scratch: ") + cudaGetErrorString(e));
            p->d_gscratch = static_cast<float2 *>(ptr);
            p->gscratch_bytes = need;
        }
    }
    for (const auto &grp : p->groups)
        if (grp.force_path >= 3) {
            const int rc = ensure_rows_scratch(p, st);
            if (rc) return rc;
            break;
        }
    // without an output array (d_adjoint set), groups whose adjoint columns
    // come from stored images image into the plan's own image array
    // (allocated on first need, before any graph capture records this call)
    float *d_tmp = nullptr;
    if (!d_images && p->n_layers) {
        bool need = false;
        for (const auto &grp : p->groups) need = need || gemm_ok(grp) || !blink::adjoint_fusable(grp.n_px);
        if (need && !p->d_imgtmp) {
            void *ptr = nullptr;
            const cudaError_t e = cudaMallocFromPoolAsync(&ptr, size_t(p->out_extent) * sizeof(float), ctx->pool, st);
            if (e != cudaSuccess)
                return fail(ctx, BLINK_ERR_WORKSPACE, std::string("plan images: ") + cudaGetErrorString(e));
            p->d_imgtmp = static_cast<float *>(ptr);
        }
        if (need) d_tmp = p->d_imgtmp;
    }
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        const auto &grp = p->groups[gi];
        float *img = d_images;
        if (!img && (gemm_ok(grp) || !blink::adjoint_fusable(grp.n_px))) img = d_tmp;
        blink::ImageArgs a = group_args(p, grp, d_vis, img, d_wsum, flags & BLINK_NORMALIZE);
        float2 *adj = d_adjoint ? reinterpret_cast<float2 *>(d_adjoint) + adjoint_offset(p, gi) : nullptr;
        a.gains = reinterpret_cast<const float2 *>(d_gains);
        a.gain_stride = epi ? epi->gain_stride : 0;
        a.gain_period = epi ? epi->gain_period : 0;
        a.gprod = gprod;
        a.ref = d_ref;
        if (d_sqnorm) {
            a.sq_part = p->d_sqpart;
            a.sq_stride = p->sq_stride;
        }
        Error e;
        if (gemm_ok(grp)) {
            a.scratch = p->d_gscratch;
            a.scratch_bytes = p->gscratch_bytes;
            e = blink::launch_dftgemm_group(grp.n_px, int(mode), a, st);
            if (!e.status && d_wsum) e = blink::launch_wsum_copy(a, st);
            // the adjoint's columns from the stored images
            if (!e.status && adj) e = blink::launch_degrid_cols_group(grp.n_px, a, img, adj, st);
        } else {
            a.adj = adj;
            e = blink::launch_image_group(grp.n_px, a, st);
        }
        if (e.status) return fail(ctx, e);
    }
    if (d_sqnorm) {
        Error e = blink::launch_sq_totals(p->d_sqpart, p->sq_stride, p->n_layers, d_sqnorm, st);
        if (e.status) return fail(ctx, e);
    }
    return BLINK_OK;
}

int blink_plan_check(blink_plan *p, void *stream) {
    if (!p) return BLINK_ERR_INVALID;
    DeviceGuard g(p->ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int word = 0;
    if (cudaMemcpyAsync(&word, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(p->d_status, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return fail(p->ctx, BLINK_ERR_CUDA, "status read failed");
    if (word) return fail(p->ctx, word, "a bounded device-side wait gave up");
    return BLINK_OK;
}

void blink_plan_destroy(blink_plan *p) {
    if (!p) return;
    {
        DeviceGuard g(p->ctx->device);
        if (p->graph) cudaGraphExecDestroy(p->graph);
        free_plan_memory(p, p->last_stream);
        if (p->cap_stream) {
            cudaStreamSynchronize(p->last_stream);
            cudaStreamDestroy(p->cap_stream);
        }
    }
    delete p;
}

int blink_plan_autotune(blink_plan *p, const float *d_vis, float *d_images, void *stream) {
    if (!p) return BLINK_ERR_INVALID;
    blink_ctx *ctx = p->ctx;
    if (p->n_layers && (!d_vis || !d_images)) return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    p->last_stream = st;
    int rc = ensure_rows_scratch(p, st);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(ctx, BLINK_ERR_CUDA, "event creation failed");
    struct Cand {
        int path;
        size_t budget;
    };
    for (auto &grp : p->groups) {
        std::vector<Cand> cands;
        if (blink::image_small_path(grp.n_px, grp.r_alloc)) {
            if (grp.sched_ok) cands.push_back({1, 0});
            cands.push_back({2, 0});
        }
        for (size_t mb : {12, 24, 48}) cands.push_back({3, mb << 20});
        for (size_t mb : {12, 24, 48}) cands.push_back({4, mb << 20});
        float best = 1e30f;
        Cand pick = cands.front();
        for (const Cand &c : cands) {
            grp.force_path = c.path;
            grp.wave_budget = c.budget;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && !rc; ++rep) {  // first run warms up
                blink::ImageArgs a = group_args(p, grp, d_vis, d_images, nullptr, 0);
                cudaEventRecord(e0, st);
                Error e = blink::launch_image_group(grp.n_px, a, st);
                cudaEventRecord(e1, st);
                if (e.status) rc = fail(ctx, e);
                else if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(ctx, BLINK_ERR_CUDA, "autotune timing failed");
                else cudaEventElapsedTime(&ms, e0, e1);
            }
            if (rc) break;
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        grp.force_path = pick.path;
        grp.wave_budget = pick.budget;
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) ctx->err.clear();
    return rc;
}

int blink_plan_tuning(const blink_plan *p, int group, int *n_px, int *path, int64_t *wave_bytes) {
    if (!p || group < 0 || group >= int(p->groups.size())) return BLINK_ERR_INVALID;
    const auto &grp = p->groups[size_t(group)];
    if (n_px) *n_px = grp.n_px;
    if (path) *path = grp.force_path;
    if (wave_bytes) *wave_bytes = int64_t(grp.wave_budget);
    return BLINK_OK;
}

int blink_ctx_set_wait_limit(blink_ctx *ctx, int64_t limit_ns) {
    if (!ctx) return BLINK_ERR_INVALID;
    ctx->wait_ns = limit_ns < 0 ? -1 : limit_ns;
    return BLINK_OK;
}

int blink_plan_set_tuning(blink_plan *p, int group, int path, int64_t wave_bytes) {
    if (!p) return BLINK_ERR_INVALID;
    if (group < 0 || group >= int(p->groups.size()))
        return fail(p->ctx, BLINK_ERR_INVALID, "size group out of range");
    auto &grp = p->groups[size_t(group)];
    const bool small = blink::image_small_path(grp.n_px, grp.r_alloc);
    if (path < 0 || path > 4 || wave_bytes < 0 || (path == 1 && !(small && grp.sched_ok)) ||
        (path == 2 && !small))
        return fail(p->ctx, BLINK_ERR_INVALID, "kernel path not available for this size group");
    grp.force_path = path;
    grp.wave_budget = size_t(wave_bytes);
    return BLINK_OK;
}

int blink_plan_capture(blink_plan *p, const float *d_vis, float *d_images, float *d_wsum, uint32_t flags,
                       const blink_epilogue *epi, void *stream) {
    if (!p) return BLINK_ERR_INVALID;
    blink_ctx *ctx = p->ctx;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every allocation happens before capture
    int rc = ensure_rows_scratch(p, st);
    if (rc) return rc;
    rc = blink_plan_image_ex(p, d_vis, d_images, d_wsum, flags, epi, stream);  // also allocates lazily
    if (rc) return rc;
    if (!p->cap_stream && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, BLINK_ERR_CUDA, "capture stream creation failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(ctx, BLINK_ERR_CUDA, "synchronise failed");
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(ctx, BLINK_ERR_CUDA, "begin capture failed");
    const cudaStream_t keep = p->last_stream;
    rc = blink_plan_image_ex(p, d_vis, d_images, d_wsum, flags, epi, p->cap_stream);
    p->last_stream = keep;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->cap_stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ec != cudaSuccess || !graph) return fail(ctx, BLINK_ERR_CUDA, "end capture failed");
    const cudaError_t ei = cudaGraphInstantiate(&p->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(ctx, BLINK_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    ctx->err.clear();
    return BLINK_OK;
}

int blink_plan_replay(blink_plan *p, void *stream) {
    if (!p) return BLINK_ERR_INVALID;
    if (!p->graph) return fail(p->ctx, BLINK_ERR_INVALID, "no captured graph (call blink_plan_capture)");
    DeviceGuard g(p->ctx->device);
    const cudaError_t e = cudaGraphLaunch(p->graph, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(p->ctx, BLINK_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    p->last_stream = static_cast<cudaStream_t>(stream);
    return BLINK_OK;
}

int blink_plan_degrid(blink_plan *p, const float *d_dimage, float *d_dvis, uint32_t flags, void *stream) {
    return blink_plan_degrid_scaled(p, d_dimage, nullptr, d_dvis, flags, stream);
}

int blink_plan_degrid_scaled(blink_plan *p, const float *d_dimage, const float *d_layer_scale, float *d_dvis,
                             uint32_t flags, void *stream) {
    if (!p) return BLINK_ERR_INVALID;
    blink_ctx *ctx = p->ctx;
    if (p->n_layers && (!d_dimage || !d_dvis)) return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    if (flags & ~uint32_t(BLINK_NORMALIZE)) return fail(ctx, BLINK_ERR_INVALID, "unknown flags");
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!p->d_dscratch && p->n_layers) {
        size_t need = 0;
        for (const auto &grp : p->groups) {
            const size_t per = blink::degrid_scratch_per_layer(grp.n_px, grp.r_alloc);
            need = std::max(need, std::max(per, std::min(per * size_t(grp.count), kScratchCap)));
        }
        void *ptr = nullptr;
        const cudaError_t e = cudaMallocFromPoolAsync(&ptr, need, ctx->pool, st);
        if (e != cudaSuccess)
            return fail(ctx, BLINK_ERR_WORKSPACE, std::string("adjoint scratch: ") + cudaGetErrorString(e));
        p->d_dscratch = static_cast<float2 *>(ptr);
        p->dscratch_bytes = need;
    }
    p->last_stream = st;
    for (const auto &grp : p->groups) {
        blink::ImageArgs a = group_args(p, grp, nullptr, nullptr, nullptr, flags);
        a.scratch = p->d_dscratch;
        a.scratch_bytes = p->dscratch_bytes;
        a.lscale = d_layer_scale;
        Error e = blink::launch_degrid_group(grp.n_px, a, d_dimage, reinterpret_cast<float2 *>(d_dvis), st);
        if (e.status) return fail(ctx, e);
    }
    return BLINK_OK;
}

int blink_plan_adjoint_bytes(const blink_plan *p, int64_t *bytes) {
    if (!p || !bytes) return BLINK_ERR_INVALID;
    *bytes = adjoint_offset(p, p->groups.size()) * int64_t(sizeof(float2));
    return BLINK_OK;
}

int blink_plan_degrid_adjoint(blink_plan *p, const float *d_adjoint, const float *d_layer_scale, float *d_dvis,
                              uint32_t flags, void *stream) {
    if (!p) return BLINK_ERR_INVALID;
    blink_ctx *ctx = p->ctx;
    if (p->n_layers && (!d_adjoint || !d_dvis)) return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    if (reinterpret_cast<uintptr_t>(d_adjoint) & 7)
        return fail(ctx, BLINK_ERR_INVALID, "adjoint buffer must be 8-byte aligned");
    if (flags & ~uint32_t(BLINK_NORMALIZE)) return fail(ctx, BLINK_ERR_INVALID, "unknown flags");
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    p->last_stream = st;
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        const auto &grp = p->groups[gi];
        blink::ImageArgs a = group_args(p, grp, nullptr, nullptr, nullptr, flags);
        a.lscale = d_layer_scale;
        const float2 *in = reinterpret_cast<const float2 *>(d_adjoint) + adjoint_offset(p, gi);
        Error e = blink::launch_degrid_rows_group(grp.n_px, a, in, reinterpret_cast<float2 *>(d_dvis), st);
        if (e.status) return fail(ctx, e);
    }
    return BLINK_OK;
}

int blink_degrid(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers, int n_layers,
                 const float *d_dimage, float *d_dvis, uint32_t flags, void *stream) {
    blink_plan *p = nullptr;
    int st = blink_plan_create(ctx, d_ant_xyz, n_ant, h_layers, n_layers, &p, stream);
    if (st) return st;
    st = blink_plan_degrid(p, d_dimage, d_dvis, flags, stream);
    blink_plan_destroy(p);
    return st;
}

// Per-layer visibility offsets of h_layers in a stream-ordered device array.
static int upload_offsets(blink_ctx *ctx, const blink_layer *h_layers, int n_layers, cudaStream_t st, int64_t **out) {
    std::vector<int64_t> off(static_cast<size_t>(n_layers));
    for (int l = 0; l < n_layers; ++l) off[size_t(l)] = h_layers[l].vis_offset;
    void *ptr = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&ptr, sizeof(int64_t) * off.size(), ctx->pool, st);
    if (e != cudaSuccess) return fail(ctx, BLINK_ERR_WORKSPACE, "offset table allocation failed");
    e = cudaMemcpyAsync(ptr, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(ptr, st);
        return fail(ctx, BLINK_ERR_CUDA, std::string("offset upload: ") + cudaGetErrorString(e));
    }
    *out = static_cast<int64_t *>(ptr);
    return BLINK_OK;
}

static int check_gain_args(blink_ctx *ctx, int n_ant, const blink_layer *h_layers, int n_layers) {
    if (!ctx) return BLINK_ERR_INVALID;
    if (n_ant < 2) return fail(ctx, BLINK_ERR_INVALID, "n_ant must be >= 2");
    if (n_layers < 0 || (n_layers && !h_layers)) return fail(ctx, BLINK_ERR_INVALID, "bad layer array");
    for (int l = 0; l < n_layers; ++l)
        if (h_layers[l].vis_offset < 0) return fail(ctx, BLINK_ERR_INVALID, "offsets must be >= 0");
    return BLINK_OK;
}

int blink_apply_gains(blink_ctx *ctx, int n_ant, const blink_layer *h_layers, int n_layers, const float *d_model,
                      const float *d_gains, float *d_vis, void *stream) {
    int st = check_gain_args(ctx, n_ant, h_layers, n_layers);
    if (st || n_layers == 0) return st;
    if (!d_model || !d_gains || !d_vis) return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t *d_off = nullptr;
    st = upload_offsets(ctx, h_layers, n_layers, s, &d_off);
    if (st) return st;
    Error e = blink::launch_apply_gains(reinterpret_cast<const float2 *>(d_model), reinterpret_cast<const float2 *>(d_gains),
                                        d_off, n_layers, n_ant, int64_t(n_ant) * (n_ant - 1) / 2,
                                        reinterpret_cast<float2 *>(d_vis), s);
    cudaFreeAsync(d_off, s);
    if (e.status) return fail(ctx, e);
    ctx->err.clear();
    return BLINK_OK;
}

int blink_gain_grad(blink_ctx *ctx, int n_ant, const blink_layer *h_layers, int n_layers, const float *d_dvis,
                    const float *d_model, const float *d_gains, float *d_dgains, void *stream) {
    int st = check_gain_args(ctx, n_ant, h_layers, n_layers);
    if (st) return st;
    if (!d_dvis || !d_model || !d_gains || !d_dgains) return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    if (n_ant > 1024) return fail(ctx, BLINK_ERR_UNSUPPORTED, "gain gradient: more than 1024 antennas");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_layers == 0) {
        const cudaError_t e = cudaMemsetAsync(d_dgains, 0, sizeof(float2) * size_t(n_ant), s);
        return e == cudaSuccess ? BLINK_OK : fail(ctx, BLINK_ERR_CUDA, "memset failed");
    }
    int64_t *d_off = nullptr;
    st = upload_offsets(ctx, h_layers, n_layers, s, &d_off);
    if (st) return st;
    void *d_part = nullptr;
    if (cudaMallocFromPoolAsync(&d_part, blink::gain_grad_scratch_bytes(n_layers, n_ant), ctx->pool, s) !=
        cudaSuccess) {
        cudaFreeAsync(d_off, s);
        return fail(ctx, BLINK_ERR_WORKSPACE, "gain-gradient scratch allocation failed");
    }
    Error e = blink::launch_gain_grad(reinterpret_cast<const float2 *>(d_dvis), reinterpret_cast<const float2 *>(d_model),
                                      reinterpret_cast<const float2 *>(d_gains), d_off, n_layers, n_ant,
                                      reinterpret_cast<float2 *>(d_dgains), d_part, s);
    cudaFreeAsync(d_part, s);
    cudaFreeAsync(d_off, s);
    if (e.status) return fail(ctx, e);
    ctx->err.clear();
    return BLINK_OK;
}

int blink_plan_layer_info(const blink_plan *p, int layer, float *wsum, int64_t *n_kept) {
    if (!p || layer < 0 || layer >= p->n_layers) return BLINK_ERR_INVALID;
    const ChanInfo &ci = p->infos[size_t(p->layer_chan[size_t(layer)])];
    if (wsum) *wsum = ci.wsum;
    if (n_kept) *n_kept = ci.n_kept;
    return BLINK_OK;
}

int blink_image_batch(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
                      int n_layers, const float *d_vis, float *d_images, float *d_wsum, uint32_t flags,
                      void *stream) {
    blink_plan *p = nullptr;
    int st = blink_plan_create(ctx, d_ant_xyz, n_ant, h_layers, n_layers, &p, stream);
    if (st) return st;
    st = blink_plan_image(p, d_vis, d_images, d_wsum, flags, stream);
    blink_plan_destroy(p);
    return st;
}

int blink_cells(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
                int n_layers, int32_t *d_cells, void *stream) {
    int st = validate(ctx, d_ant_xyz, n_ant, h_layers, n_layers);
    if (st) return st;
    if (n_layers && !d_cells) return fail(ctx, BLINK_ERR_INVALID, "d_cells is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    blink_plan p;
    st = build_plan(ctx, d_ant_xyz, n_ant, h_layers, n_layers, true, &p, s);
    if (!st) {
        Error e = blink::launch_expand_cells(p.d_cells, p.d_layers, n_layers, p.nb,
                                             reinterpret_cast<int2 *>(d_cells), s);
        if (e.status) st = fail(ctx, e);
    }
    free_plan_memory(&p, s);
    if (!st) ctx->err.clear();
    return st;
}

int blink_grid(blink_ctx *ctx, const double *d_ant_xyz, int n_ant, const blink_layer *h_layers,
               int n_layers, const float *d_vis, float *d_grid, float *d_wsum, void *stream) {
    int st = validate(ctx, d_ant_xyz, n_ant, h_layers, n_layers);
    if (st) return st;
    if (n_layers && (!d_vis || !d_grid)) return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    blink_plan p;
    st = build_plan(ctx, d_ant_xyz, n_ant, h_layers, n_layers, false, &p, s);
    if (!st) {
        for (const auto &grp : p.groups) {
            Error e = blink::launch_grid_group(grp.n_px, group_args(&p, grp, d_vis, d_grid, d_wsum, 0), s);
            if (e.status) {
                st = fail(ctx, e);
                break;
            }
        }
    }
    free_plan_memory(&p, s);
    if (!st) ctx->err.clear();
    return st;
}


// ------------------------------------------------------------ host buffers
}  // extern "C"

namespace {

// Resources of one blink_image_batch_host call (released by host_release).
struct HostPipe {
    double *d_xyz = nullptr;
    float2 *d_vis[2] = {nullptr, nullptr};
    float *d_out[2] = {nullptr, nullptr};
    float *d_ws = nullptr;
    DevLayer *d_cl = nullptr;
    blink_plan plan;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
};

struct HostChunk {
    int l0, l1;
    int64_t vis_base, vis_end, out_base, out_end;
};

struct HostGroup {
    int chunk, n_px, first, count, r_alloc, sched_ok, max_chunk, max_seg;
};

#define HTRY(call)                                                                                   \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(ctx, BLINK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

int host_pipeline(blink_ctx *ctx, HostPipe &hp, const double *h_ant_xyz, int n_ant, const blink_layer *h_layers,
                  int n_layers, const float *h_vis, float *h_images, float *h_wsum, uint32_t flags,
                  cudaStream_t s) {
    const int64_t nb = int64_t(n_ant) * (n_ant - 1) / 2;
    // chunks of consecutive layers bounded by the staging sizes
    const size_t cap_vis = size_t(128) << 20, cap_out = size_t(128) << 20;  // 128 MB: shorter fill and drain of the copy pipeline
    std::vector<HostChunk> chunks;
    for (int l = 0; l < n_layers;) {
        HostChunk c{l, l, INT64_MAX, 0, INT64_MAX, 0};
        while (c.l1 < n_layers && c.l1 - c.l0 < 65535) {
            const blink_layer &L = h_layers[c.l1];
            const int64_t vb = std::min(c.vis_base, L.vis_offset), ve = std::max(c.vis_end, L.vis_offset + nb);
            const int64_t ob = std::min(c.out_base, L.out_offset);
            const int64_t oe = std::max(c.out_end, L.out_offset + int64_t(L.n_px) * L.n_px);
            if (c.l1 > c.l0 && (size_t(ve - vb) * 8 > cap_vis || size_t(oe - ob) * 4 > cap_out)) break;
            c.vis_base = vb, c.vis_end = ve, c.out_base = ob, c.out_end = oe;
            ++c.l1;
        }
        chunks.push_back(c);
        l = c.l1;
    }
    size_t need_vis = 0, need_out = 0;
    for (auto &c : chunks) {
        need_vis = std::max(need_vis, size_t(c.vis_end - c.vis_base) * 8);
        need_out = std::max(need_out, size_t(c.out_end - c.out_base) * 4);
    }
    const int nbuf = chunks.size() > 1 ? 2 : 1;
    auto alloc = [&](void **ptr, size_t bytes) {
        return cudaMallocFromPoolAsync(ptr, std::max<size_t>(bytes, 256), ctx->pool, s) == cudaSuccess;
    };
    bool ok = alloc(reinterpret_cast<void **>(&hp.d_xyz), sizeof(double) * 3 * size_t(n_ant)) &&
              alloc(reinterpret_cast<void **>(&hp.d_ws), sizeof(float) * size_t(n_layers));
    for (int b = 0; b < nbuf && ok; ++b)
        ok = alloc(reinterpret_cast<void **>(&hp.d_vis[b]), need_vis) &&
             alloc(reinterpret_cast<void **>(&hp.d_out[b]), need_out);
    if (!ok) return fail(ctx, BLINK_ERR_WORKSPACE, "staging allocation failed");
    for (int b = 0; b < 2; ++b) {
        HTRY(cudaEventCreateWithFlags(&hp.ev_in[b], cudaEventDisableTiming));
        HTRY(cudaEventCreateWithFlags(&hp.ev_comp[b], cudaEventDisableTiming));
        HTRY(cudaEventCreateWithFlags(&hp.ev_out[b], cudaEventDisableTiming));
    }
    // The first chunks' visibilities need only the staging buffers: their
    // copies start now and overlap the plan build (uv, cells, tables).
    auto copy_in = [&](int ci) -> int {
        const HostChunk &c = chunks[size_t(ci)];
        const int b = ci % nbuf;
        if (ci >= nbuf) HTRY(cudaStreamWaitEvent(ctx->copy_in, hp.ev_comp[b], 0));  // vis buffer free
        HTRY(cudaMemcpyAsync(hp.d_vis[b], h_vis + 2 * c.vis_base, size_t(c.vis_end - c.vis_base) * 8,
                             cudaMemcpyHostToDevice, ctx->copy_in));
        HTRY(cudaEventRecord(hp.ev_in[b], ctx->copy_in));
        return BLINK_OK;
    };
    HTRY(cudaEventRecord(hp.ev_out[0], s));  // staging allocated on s
    HTRY(cudaStreamWaitEvent(ctx->copy_in, hp.ev_out[0], 0));
    const int early = std::min<int>(nbuf, int(chunks.size()));
    for (int ci = 0; ci < early; ++ci)
        if (int e = copy_in(ci)) return e;
    HTRY(cudaMemcpyAsync(hp.d_xyz, h_ant_xyz, sizeof(double) * 3 * size_t(n_ant), cudaMemcpyHostToDevice, s));
    int st = build_plan(ctx, hp.d_xyz, n_ant, h_layers, n_layers, false, &hp.plan, s);
    if (st) return st;
    const blink_plan &p = hp.plan;
    // per chunk: layers rebased onto the staging buffers, grouped by size
    std::vector<DevLayer> cl;
    std::vector<HostGroup> groups;
    for (int ci = 0; ci < int(chunks.size()); ++ci) {
        const HostChunk &c = chunks[size_t(ci)];
        std::vector<int> idx;
        for (int l = c.l0; l < c.l1; ++l) idx.push_back(l);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return h_layers[x].n_px < h_layers[y].n_px; });
        for (int l : idx) {
            const int ch = p.layer_chan[size_t(l)];
            const ChanInfo &inf = p.infos[size_t(ch)];
            if (groups.empty() || groups.back().chunk != ci || groups.back().n_px != h_layers[l].n_px)
                groups.push_back(HostGroup{ci, h_layers[l].n_px, int(cl.size()), 0, 1, 1, 0, 0});
            HostGroup &gg = groups.back();
            gg.count++;
            gg.r_alloc = std::max(gg.r_alloc, inf.rows);
            gg.sched_ok = gg.sched_ok && p.d_sched && inf.sched_off >= 0 && inf.sched == 1;
            gg.max_chunk = std::max(gg.max_chunk, inf.chunk);
            gg.max_seg = std::max(gg.max_seg, inf.max_seg);
            cl.push_back(DevLayer{h_layers[l].vis_offset - c.vis_base, h_layers[l].out_offset - c.out_base, ch, l});
        }
    }
    if (!alloc(reinterpret_cast<void **>(&hp.d_cl), sizeof(DevLayer) * cl.size()))
        return fail(ctx, BLINK_ERR_WORKSPACE, "layer table allocation failed");
    HTRY(cudaMemcpyAsync(hp.d_cl, cl.data(), sizeof(DevLayer) * cl.size(), cudaMemcpyHostToDevice, s));
    // plan and layer table are ready on s before any image copy-out
    HTRY(cudaEventRecord(hp.ev_out[1], s));
    HTRY(cudaStreamWaitEvent(ctx->copy_out, hp.ev_out[1], 0));
    size_t gi = 0;
    for (int ci = 0; ci < int(chunks.size()); ++ci) {
        const HostChunk &c = chunks[size_t(ci)];
        const int b = ci % nbuf;
        if (ci >= early)
            if (int e = copy_in(ci)) return e;
        HTRY(cudaStreamWaitEvent(s, hp.ev_in[b], 0));
        if (ci >= nbuf) HTRY(cudaStreamWaitEvent(s, hp.ev_out[b], 0));  // image buffer drained
        for (; gi < groups.size() && groups[gi].chunk == ci; ++gi) {
            const HostGroup &gg = groups[gi];
            blink_plan::Group grp{gg.n_px, 0, gg.count, gg.r_alloc, gg.sched_ok, gg.max_chunk, gg.max_seg};
            blink::ImageArgs a =
                group_args(&p, grp, reinterpret_cast<const float *>(hp.d_vis[b]), hp.d_out[b], hp.d_ws, flags);
            a.layers = hp.d_cl + gg.first;
            Error e = blink::launch_image_group(gg.n_px, a, s);
            if (e.status) return fail(ctx, e);
        }
        HTRY(cudaEventRecord(hp.ev_comp[b], s));
        HTRY(cudaStreamWaitEvent(ctx->copy_out, hp.ev_comp[b], 0));
        HTRY(cudaMemcpyAsync(h_images + c.out_base, hp.d_out[b], size_t(c.out_end - c.out_base) * 4,
                             cudaMemcpyDeviceToHost, ctx->copy_out));
        HTRY(cudaEventRecord(hp.ev_out[b], ctx->copy_out));
    }
    if (h_wsum) HTRY(cudaMemcpyAsync(h_wsum, hp.d_ws, sizeof(float) * size_t(n_layers), cudaMemcpyDeviceToHost, s));
    HTRY(cudaEventRecord(hp.ev_in[0], ctx->copy_out));
    HTRY(cudaStreamWaitEvent(s, hp.ev_in[0], 0));
    return BLINK_OK;
}
#undef HTRY

// Frees everything on s after the pipeline (or whatever part of it ran).
int host_release(blink_ctx *ctx, HostPipe &hp, cudaStream_t s, int st) {
    // whatever was queued on the copy streams must finish before the frees
    cudaEvent_t fin = nullptr;
    if (cudaEventCreateWithFlags(&fin, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(fin, ctx->copy_in);
        cudaStreamWaitEvent(s, fin, 0);
        cudaEventRecord(fin, ctx->copy_out);
        cudaStreamWaitEvent(s, fin, 0);
    }
    free_plan_memory(&hp.plan, s);
    for (void *ptr : {static_cast<void *>(hp.d_xyz), static_cast<void *>(hp.d_ws), static_cast<void *>(hp.d_cl)})
        if (ptr) cudaFreeAsync(ptr, s);
    if (hp.d_vis[0]) cudaFreeAsync(hp.d_vis[0], s);
    if (hp.d_out[0]) cudaFreeAsync(hp.d_out[0], s);
    if (hp.d_vis[1]) cudaFreeAsync(hp.d_vis[1], s);
    if (hp.d_out[1]) cudaFreeAsync(hp.d_out[1], s);
    const cudaError_t se = cudaStreamSynchronize(s);
    if (fin) cudaEventDestroy(fin);
    for (int b = 0; b < 2; ++b) {
        if (hp.ev_in[b]) cudaEventDestroy(hp.ev_in[b]);
        if (hp.ev_comp[b]) cudaEventDestroy(hp.ev_comp[b]);
        if (hp.ev_out[b]) cudaEventDestroy(hp.ev_out[b]);
    }
    if (!st && se != cudaSuccess) st = fail(ctx, BLINK_ERR_CUDA, std::string("pipeline: ") + cudaGetErrorString(se));
    return st;
}

}  // namespace

extern "C" {

// Chunked pipeline: H2D of chunk i+1 and D2H of chunk i-1 overlap the image
// kernels of chunk i (double-buffered device staging from the context pool).
int blink_image_batch_host(blink_ctx *ctx, const double *h_ant_xyz, int n_ant, const blink_layer *h_layers,
                           int n_layers, const float *h_vis, float *h_images, float *h_wsum, uint32_t flags,
                           void *stream) {
    if (!ctx) return BLINK_ERR_INVALID;
    int st = validate(ctx, h_ant_xyz, n_ant, h_layers, n_layers);
    if (st) return st;
    if (n_layers == 0) return BLINK_OK;
    if (!h_vis || !h_images) return fail(ctx, BLINK_ERR_INVALID, "null data pointer");
    if (flags & ~uint32_t(BLINK_NORMALIZE)) return fail(ctx, BLINK_ERR_INVALID, "unknown flags");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!ctx->copy_in && cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, BLINK_ERR_CUDA, "copy stream creation failed");
    if (!ctx->copy_out && cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, BLINK_ERR_CUDA, "copy stream creation failed");
    HostPipe hp;
    st = host_pipeline(ctx, hp, h_ant_xyz, n_ant, h_layers, n_layers, h_vis, h_images, h_wsum, flags, s);
    st = host_release(ctx, hp, s, st);
    if (!st) ctx->err.clear();
    return st;
}

}  // extern "C"
