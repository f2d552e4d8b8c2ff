// blink_noalloc.cu -- dirty images without any device memory allocation.
//
// Some callers cannot allocate device memory while they run: a real-time
// telescope pipeline that reserves all GPU memory when an observation starts
// and forbids allocation (and its latency) afterwards, or a host framework
// whose own allocator already owns the whole device.  For them this file
// provides blink_image_batch_noalloc: the imaging kernels of
// blink_image_batch, with every piece of scratch (channel tables, layer
// descriptors, gridding schedules and row buckets, the work queue, the
// row-transform ring of large images) carved out of one file-scope static
// device array of BLINK_NOALLOC_SCRATCH_BYTES bytes.  It calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// The array exists once per GPU that loads the library and lives until the
// process exits.  Every call reuses it: what must start at zero is cleared on
// each call, and calls whose work overlaps on the GPU (different streams or
// host threads at the same time) race on it.
#include "blink.h"
#include "blink_common.cuh"
#include "blink_kernels.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

using blink::ChanGeom;
using blink::ChanInfo;
using blink::DevLayer;

namespace {

constexpr size_t kBytes = BLINK_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxChannels = BLINK_NOALLOC_MAX_CHANNELS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kBytes];

// Host-side device address of g_scratch, looked up once per device.
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return BLINK_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return BLINK_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return BLINK_OK;
}

int say(char *msg, size_t cap, int status, const char *text) {
    if (msg && cap) std::snprintf(msg, cap, "%s", text);
    return status;
}

size_t up(size_t x) { return (x + 255) / 256 * 256; }

bool same_channel(const blink_layer &a, const ChanGeom &g) {
    return a.n_px == g.n_px && a.weighting == g.weighting &&
           std::memcmp(&a.freq_hz, &g.freq_hz, 8) == 0 && std::memcmp(&a.delta_u, &g.delta_u, 8) == 0;
}

// Caller's layer descriptors -> device work items (channel by exact match).
__global__ void k_layers(const blink_layer *__restrict__ raw, int n, const ChanGeom *__restrict__ geom,
                         int n_chan, DevLayer *__restrict__ out) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const blink_layer L = raw[l];
    int ch = 0;
    for (int c = 0; c < n_chan; ++c) {
        const ChanGeom g = geom[c];
        if (L.n_px == g.n_px && L.weighting == g.weighting &&
            __double_as_longlong(L.freq_hz) == __double_as_longlong(g.freq_hz) &&
            __double_as_longlong(L.delta_u) == __double_as_longlong(g.delta_u)) {
            ch = c;
            break;
        }
    }
    out[l] = DevLayer{L.vis_offset, L.out_offset, ch, l};
}

}  // namespace

extern "C" BLINK_API int blink_image_batch_noalloc(const double *d_ant_xyz, int n_ant,
                                                   const blink_layer *h_layers, int n_layers,
                                                   const float *d_vis, float *d_images, float *d_wsum,
                                                   uint32_t flags, void *stream, char *err_msg,
                                                   size_t err_cap) {
    if (err_msg && err_cap) err_msg[0] = '\0';
    if (n_layers == 0) return BLINK_OK;
    if (n_ant < 2 || !d_ant_xyz || n_layers < 0 || !h_layers || !d_vis || !d_images)
        return say(err_msg, err_cap, BLINK_ERR_INVALID, "bad array, layer or data argument");
    if (flags & ~uint32_t(BLINK_NORMALIZE)) return say(err_msg, err_cap, BLINK_ERR_INVALID, "unknown flags");
    const int64_t nb = int64_t(n_ant) * (n_ant - 1) / 2;
    const int n_px = h_layers[0].n_px;
    // distinct channels in a fixed-size host array (no heap)
    ChanGeom geoms[kMaxChannels];
    ChanInfo infos[kMaxChannels];
    int n_chan = 0, prev = -1;
    for (int l = 0; l < n_layers; ++l) {
        const blink_layer &L = h_layers[l];
        if (L.n_px != n_px)
            return say(err_msg, err_cap, BLINK_ERR_INVALID, "all layers of one call must share n_px");
        if (!blink::image_size_supported(L.n_px))
            return say(err_msg, err_cap, BLINK_ERR_UNSUPPORTED, "image size not supported");
        if ((L.weighting != BLINK_NATURAL && L.weighting != BLINK_UNIFORM) ||
            !(std::isfinite(L.freq_hz) && L.freq_hz > 0) || !(std::isfinite(L.delta_u) && L.delta_u > 0) ||
            L.vis_offset < 0 || L.out_offset < 0)
            return say(err_msg, err_cap, BLINK_ERR_INVALID, "bad layer descriptor");
        if (prev >= 0 && same_channel(L, geoms[prev])) continue;
        int c = 0;
        while (c < n_chan && !same_channel(L, geoms[c])) ++c;
        if (c == n_chan) {
            if (n_chan == kMaxChannels)
                return say(err_msg, err_cap, BLINK_ERR_WORKSPACE, "more distinct channels than the static limit");
            geoms[n_chan++] = ChanGeom{L.freq_hz, L.delta_u, L.n_px, L.weighting};
        }
        prev = c;
    }
    // layout of the static scratch: the tables blink_image_batch builds (cell
    // codes, weights, the register schedule of sizes <= 256, the row buckets
    // of large sizes), the work queue and status word, then the row-transform
    // ring of large images and, at the end, their compact grids.  A schedule or bucket set that does not fit is
    // left out and the kernels take their atomic fallback for that call.
    // the register schedule: sizes <= 256, and larger sizes whose compact
    // support is sure to fit (as blink_image_batch decides, from the array's
    // extent)
    bool large_sched = false;
    if (n_px > 256) {
        double hx[3 * 2048];
        const bool fits_host = n_ant <= 2048;
        if (fits_host && cudaMemcpyAsync(hx, d_ant_xyz, sizeof(double) * 3 * size_t(n_ant), cudaMemcpyDeviceToHost,
                                         static_cast<cudaStream_t>(stream)) == cudaSuccess &&
            cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) == cudaSuccess) {
            double x0 = hx[0], x1 = hx[0], y0 = hx[1], y1 = hx[1];
            for (int a = 1; a < n_ant; ++a) {
                x0 = std::min(x0, hx[3 * a]);
                x1 = std::max(x1, hx[3 * a]);
                y0 = std::min(y0, hx[3 * a + 1]);
                y1 = std::max(y1, hx[3 * a + 1]);
            }
            large_sched = true;
            for (int c = 0; c < n_chan && large_sched; ++c)
                large_sched = blink::cg_bound_fits(x1 - x0, y1 - y0, geoms[c].freq_hz, geoms[c].delta_u, n_px);
        }
    }
    const bool want_sched = n_px <= 256 || large_sched;
    const bool want_csr = !blink::image_small_path(n_px, n_px / 2 + 1);
    const int q_chunks = int((nb + blink::kSchedMaxChunk - 1) / blink::kSchedMaxChunk);
    int k_chunk = int((nb + q_chunks - 1) / q_chunks);
    k_chunk += k_chunk & 1;
    const size_t sched_per = want_sched ? size_t(blink::SchedLayout(n_px, nb, q_chunks).bytes) : 0;
    const size_t csr_per = want_csr ? size_t(blink::CsrLayout(n_px, nb).bytes) : 0;
    auto tables_end = [&](bool sched, bool csr) {
        const int64_t wgt_cells = int64_t(n_px / 2) * n_px;
        int64_t w = 0;
        for (int c = 0; c < n_chan; ++c)
            if (geoms[c].weighting == BLINK_UNIFORM || sched) w += wgt_cells;
        size_t o = 0;
        o = up(o + sizeof(ChanGeom) * n_chan);
        o = up(o + sizeof(ChanInfo) * n_chan);
        o = up(o + sizeof(blink_layer) * size_t(n_layers));
        o = up(o + sizeof(DevLayer) * size_t(n_layers));
        o = up(o + sizeof(uint32_t) * size_t(n_chan) * size_t(nb));
        o = up(o + sizeof(float) * size_t(w > 0 ? w : 1));
        o = up(o + sizeof(int));                                   // status word
        o = up(o + blink::image_queue_bytes(n_layers));
        if (csr) o = up(o + csr_per * n_chan);
        if (sched) o = up(o + sched_per * n_chan);
        return o;
    };
    bool use_sched = want_sched, use_csr = want_csr;
    if (use_sched && tables_end(true, use_csr) > kBytes) use_sched = false;
    if (use_csr && tables_end(use_sched, true) > kBytes) use_csr = false;
    int64_t wgt_total = 0, sched_total = 0, csr_total = 0;
    bool any_counts = false;
    for (int c = 0; c < n_chan; ++c) {
        ChanInfo ci{};
        ci.n_px = geoms[c].n_px;
        ci.weighting = geoms[c].weighting;
        ci.code_off = int64_t(c) * nb;
        ci.wgt_off = -1;
        ci.sched_off = -1;
        ci.csr_off = -1;
        if (use_sched) {
            ci.sched_large = n_px > 256 ? 1 : 0;
            ci.n_chunks = q_chunks;
            ci.chunk = k_chunk;
            ci.sched_off = sched_total;
            sched_total += int64_t(sched_per);
        }
        if (use_csr) {
            ci.csr_off = csr_total;
            csr_total += int64_t(csr_per);
        }
        if (ci.weighting == BLINK_UNIFORM || use_sched) {
            ci.wgt_off = wgt_total;
            wgt_total += int64_t(n_px / 2) * n_px;
            any_counts = true;
        }
        infos[c] = ci;
    }
    size_t off = 0;
    const size_t o_geom = off; off = up(off + sizeof(ChanGeom) * n_chan);
    const size_t o_info = off; off = up(off + sizeof(ChanInfo) * n_chan);
    const size_t o_raw = off; off = up(off + sizeof(blink_layer) * size_t(n_layers));
    const size_t o_layers = off; off = up(off + sizeof(DevLayer) * size_t(n_layers));
    const size_t o_codes = off; off = up(off + sizeof(uint32_t) * size_t(n_chan) * size_t(nb));
    const size_t o_wgt = off; off = up(off + sizeof(float) * size_t(wgt_total > 0 ? wgt_total : 1));
    const size_t o_status = off; off = up(off + sizeof(int));
    const size_t o_queue = off; off = up(off + blink::image_queue_bytes(n_layers));
    const size_t o_csr = off; off = up(off + size_t(csr_total));
    const size_t o_sched = off; off = up(off + size_t(sched_total));
    const size_t o_rows = off;
    if (off > kBytes)
        return say(err_msg, err_cap, BLINK_ERR_WORKSPACE,
                   "request needs more than BLINK_NOALLOC_SCRATCH_BYTES of tables");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return say(err_msg, err_cap, BLINK_ERR_CUDA, "no current device");
    void *base_v = nullptr;
    int st = scratch_address(dev, &base_v);
    if (st) return say(err_msg, err_cap, st, "cudaGetSymbolAddress of the static scratch failed");
    unsigned char *base = static_cast<unsigned char *>(base_v);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ChanGeom *d_geom = reinterpret_cast<ChanGeom *>(base + o_geom);
    ChanInfo *d_info = reinterpret_cast<ChanInfo *>(base + o_info);
    blink_layer *d_raw = reinterpret_cast<blink_layer *>(base + o_raw);
    DevLayer *d_layers = reinterpret_cast<DevLayer *>(base + o_layers);
    uint32_t *d_codes = reinterpret_cast<uint32_t *>(base + o_codes);
    float *d_wgt = reinterpret_cast<float *>(base + o_wgt);
    int *d_status = reinterpret_cast<int *>(base + o_status);
    int *d_queue = reinterpret_cast<int *>(base + o_queue);
    unsigned char *d_csr = csr_total ? base + o_csr : nullptr;
    unsigned char *d_sched = sched_total ? base + o_sched : nullptr;
    float2 *d_rows = reinterpret_cast<float2 *>(base + o_rows);
#define NA_TRY(call)                                                                      \
    do {                                                                                  \
        if ((call) != cudaSuccess) return say(err_msg, err_cap, BLINK_ERR_CUDA, #call);   \
    } while (0)
    NA_TRY(cudaMemcpyAsync(d_geom, geoms, sizeof(ChanGeom) * n_chan, cudaMemcpyHostToDevice, s));
    NA_TRY(cudaMemcpyAsync(d_info, infos, sizeof(ChanInfo) * n_chan, cudaMemcpyHostToDevice, s));
    NA_TRY(cudaMemcpyAsync(d_raw, h_layers, sizeof(blink_layer) * size_t(n_layers), cudaMemcpyHostToDevice, s));
    k_layers<<<(n_layers + 255) / 256, 256, 0, s>>>(d_raw, n_layers, d_geom, n_chan, d_layers);
    NA_TRY(cudaGetLastError());
    // the array keeps the last call's contents: clear everything that is accumulated
    if (any_counts) NA_TRY(cudaMemsetAsync(d_wgt, 0, sizeof(float) * size_t(wgt_total), s));
    NA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));
    if (d_csr) NA_TRY(cudaMemsetAsync(d_csr, 0, size_t(csr_total), s));
    if (d_sched) NA_TRY(cudaMemsetAsync(d_sched, 0, size_t(sched_total), s));
    blink::Error e = blink::launch_tables(d_ant_xyz, n_ant, nb, n_chan, d_geom, d_info, d_codes, nullptr,
                                          d_wgt, any_counts, s, d_sched, d_csr);
    if (e.status) return say(err_msg, err_cap, e.status, e.msg.c_str());
    NA_TRY(cudaMemcpyAsync(infos, d_info, sizeof(ChanInfo) * n_chan, cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
#undef NA_TRY
    int r_alloc = 1, max_chunk = 0, max_seg = 0, kmax = 0, row_entries = 0;
    bool sched_ok = d_sched != nullptr;
    for (int c = 0; c < n_chan; ++c) {
        r_alloc = infos[c].rows > r_alloc ? infos[c].rows : r_alloc;
        sched_ok = sched_ok && infos[c].sched_off >= 0 && infos[c].sched == 1;
        max_chunk = infos[c].chunk > max_chunk ? infos[c].chunk : max_chunk;
        max_seg = infos[c].max_seg > max_seg ? infos[c].max_seg : max_seg;
        kmax = infos[c].kmax_u > kmax ? infos[c].kmax_u : kmax;
        const int per_row = int(infos[c].n_kept / (infos[c].rows > 1 ? infos[c].rows : 1));
        row_entries = per_row > row_entries ? per_row : row_entries;
    }
    const size_t per_layer = blink::image_scratch_per_layer(n_px, r_alloc);
    size_t rows_bytes = kBytes - o_rows;
    if (per_layer > rows_bytes)
        return say(err_msg, err_cap, BLINK_ERR_WORKSPACE,
                   "one layer's row-transform buffer does not fit in BLINK_NOALLOC_SCRATCH_BYTES");
    // compact grids (as blink_image_batch uses them) at the end of the array,
    // when at least one layer's grid fits beside one layer's row buffer
    float2 *d_cg = nullptr;
    int64_t cg_stride = 0;
    int cg_cap = 0;
    if (per_layer && d_csr && blink::cg_fits(r_alloc, kmax) && rows_bytes > per_layer + 256) {
        cg_stride = (blink::cg_cells(r_alloc, kmax) + 1) & ~int64_t(1);
        const size_t per_cg = size_t(8 * cg_stride);
        const size_t fit = (rows_bytes - per_layer - 256) / per_cg;  // 256: the alignment below
        cg_cap = int(fit < size_t(n_layers) ? fit : size_t(n_layers));
        if (cg_cap >= 1) {
            const size_t cg_off = (kBytes - size_t(cg_cap) * per_cg) / 256 * 256;
            d_cg = reinterpret_cast<float2 *>(base + cg_off);
            rows_bytes = cg_off - o_rows;
        }
    }
    blink::ImageArgs a{};
    a.vis = reinterpret_cast<const float2 *>(d_vis);
    a.out = d_images;
    a.wsum_out = d_wsum;
    a.layers = d_layers;
    a.n_layers = n_layers;
    a.chans = d_info;
    a.codes = d_codes;
    a.wgt = d_wgt;
    a.nb = nb;
    a.flags = flags;
    a.r_alloc = r_alloc;
    a.scratch = per_layer ? d_rows : nullptr;
    a.scratch_bytes = per_layer ? rows_bytes : 0;
    a.sched = d_sched;
    a.sched_ok = sched_ok ? 1 : 0;
    a.max_chunk = max_chunk;
    a.max_seg = max_seg;
    a.status = d_status;
    a.csr = d_csr;
    a.csr_bytes = size_t(csr_total);
    a.kmax = kmax;
    a.row_entries = row_entries;
    a.n_ant = n_ant;
    a.queue = d_queue;
    a.queue_bytes = blink::image_queue_bytes(n_layers);
    if (d_cg) {
        a.cg = d_cg;
        a.cg_stride = cg_stride;
        a.cg_cap = cg_cap;
    }
    e = blink::launch_image_group(n_px, a, s);
    if (e.status) return say(err_msg, err_cap, e.status, e.msg.c_str());
    return BLINK_OK;
}
