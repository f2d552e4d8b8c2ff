// blink_kernels.cuh -- host-side launchers of the library's kernels.
#pragma once

#include "blink_common.cuh"

namespace blink {

// uv, cells and weighting tables for n_chan channels (blink_tables.cu).
// info[] must hold n_px, weighting, code_off, wgt_off, the schedule fields
// and zeroed accumulators; channels with wgt_off >= 0 must have (N/2)*N
// zeroed int32 counts at wgt + wgt_off (they become 1/n weights for uniform
// weighting).
// sched (may be null): per-channel schedule blocks at ChanInfo::sched_off,
// zeroed, for channels imaged by the register-accumulation gridding.
Error launch_tables(const double *ant_xyz, int n_ant, int64_t nb, int n_chan, const ChanGeom *geom,
                    ChanInfo *info, uint32_t *codes, int2 *cells, float *wgt, bool any_counts,
                    cudaStream_t st, unsigned char *sched = nullptr, unsigned char *csr = nullptr);
Error launch_expand_cells(const int2 *cells, const DevLayer *layers, int n_layers, int64_t nb,
                          int2 *out, cudaStream_t st);

// Arguments shared by the gridding / imaging launchers (blink_image.cu).
struct ImageArgs {
    const float2 *vis;          // visibilities, complex64
    void *out;                  // images (float) or grids (float2)
    float *wsum_out;            // [caller layers] or null
    const DevLayer *layers;     // this group's layers (device)
    int n_layers;               // layers in the group
    const ChanInfo *chans;      // device channel table
    const uint32_t *codes;      // packed canonical cells
    const float *wgt;           // uniform weights
    int64_t nb;                 // baselines per layer
    uint32_t flags;             // BLINK_NORMALIZE ...
    int r_alloc;                // max support rows over the group's channels
    float2 *scratch;            // large-image row-transform buffer (or null)
    size_t scratch_bytes;
    const unsigned char *sched; // register-accumulation schedules (or null)
    int sched_ok;               // every channel of the group has a schedule
    int max_chunk;              // largest staging chunk of the group's channels
    int max_seg;                // longest per-chunk schedule segment (entries)
    int *status;                // device status word (bounded waits report BLINK_ERR_TIMEOUT)
    const unsigned char *csr;   // row buckets of large-image channels (or null)
    int force_path;             // 0 default, 1 scheduled fused, 2 atomic fused, 3 persistent queue, 4 waves
    size_t wave_budget;         // row-transform scratch per wave (0 = default, L2-sized)
    // fused epilogue (all null/0 when unused)
    const float2 *gains;        // antenna gains; layer l uses row (l mod gain_period, or l)
    int64_t gain_stride;        // complex elements between gain rows
    int64_t gain_period;        // 0 = no wrap
    int n_ant;                  // antennas (baseline b <-> pair, for the gains)
    const float2 *gprod;        // gain products g_i conj(g_j) [gain rows][nb], or null
                                // (then the kernels form them from `gains`)
    const float *ref;           // reference images, addressed like the output
    int64_t wait_ns = -1;       // first-wait limit of the tensor-core kernels (< 0: default 1 s)
    int kmax = 0;               // max |k_u| of the group's channels (compact support of pass 1)
    // optional second stream for the adjoint's waves (forked from and joined
    // back to the launch stream with these two events); null: one stream
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // work queue of the persistent large-image kernel (device words, zeroed by
    // the launcher); null: the large-image path runs in waves of two kernels
    int *queue = nullptr;
    size_t queue_bytes = 0;
    size_t csr_bytes = 0;       // row buckets of all channels (the large kernel looks ahead
                                // for them only when they cannot all stay in L2)
    int row_entries = 0;        // largest kept baselines per support row among the group's
                                // channels (sets the band height of large-image row items)
    // compact grids of large-image layers (k_grid_compact): when set, the row
    // items read their rows from cg instead of gathering visibilities.  cg
    // holds cg_cap layers of cg_stride complex elements; slot s is layer
    // cg_l0 + s of `layers` (the launchers fill it wave by wave)
    float2 *cg = nullptr;
    int64_t cg_stride = 0;
    int cg_cap = 0;
    int cg_l0 = 0;
    // fused epilogue's per-layer sum of squares of the output: the kernels
    // write partial sums to sq_part[caller layer * sq_stride + slot] (slot =
    // column item; slots a size does not use are zeroed), launch_sq_totals
    // adds each row in slot order.  Null: not computed.
    double *sq_part = nullptr;
    int sq_stride = 0;
    // adjoint: per caller layer factor on the visibility gradient (or null)
    const float *lscale = nullptr;
    // fused epilogue: the adjoint's column transforms of the stored output,
    // r_alloc rows of N complex per layer of the group (or null)
    float2 *adj = nullptr;
};

// Compact gridding (blink_compact.cu) of layers [l0, l0 + cnt) of a.layers
// into a.cg slots 0 .. cnt - 1 (cnt <= a.cg_cap; the group's channels need
// row buckets and cg_fits), and the shared memory it takes.
Error launch_grid_compact(const ImageArgs &a, int l0, int cnt, cudaStream_t st);
size_t grid_compact_smem(int64_t cg_stride);

// Device words the persistent large-image kernel needs for a group of
// n_layers layers (its work queue and per-layer counters).
size_t image_queue_bytes(int n_layers);

// Per-size launchers (defined in blink_image_impl.cuh, instantiated once per
// size in the blink_image_<sizes>.cu units).
template <int N>
struct SizeOps {
    static Error image(const ImageArgs &a, cudaStream_t st);
    static Error rows_wave(const ImageArgs &a, int l0, int cnt, cudaStream_t st);
    static Error degrid(const ImageArgs &a, const float *resid, float2 *dvis, cudaStream_t st);
    static Error degrid_rows(const ImageArgs &a, const float2 *in, float2 *dvis, cudaStream_t st);
    static Error degrid_cols(const ImageArgs &a, const float *resid, float2 *out, cudaStream_t st);
    static bool small(int r_alloc);
    static size_t scratch_per_layer(int r_alloc);
    static int sq_slots();
    static bool adj_fusable();
};

bool image_size_supported(int n_px);
int supported_sizes(int32_t *out, int cap);
// Bytes of row-transform scratch one layer of size n_px with r_alloc rows needs
// on the large-image path (0 if the fused single-CTA path takes the group).
size_t image_scratch_per_layer(int n_px, int r_alloc);
// Whether the fused single-CTA kernels can take a group, and the scratch a
// layer needs on the two-kernel path regardless of that choice.
bool image_small_path(int n_px, int r_alloc);
size_t image_rows_scratch_per_layer(int n_px, int r_alloc);
Error launch_image_group(int n_px, const ImageArgs &a, cudaStream_t st);
Error launch_grid_group(int n_px, const ImageArgs &a, cudaStream_t st);
Error launch_wsum_copy(const ImageArgs &a, cudaStream_t st);

// Pass 1 only (gridding + row transforms) for layers [l0, l0 + cnt) of a
// group into scratch[l - l0][r][p] (natural order, FP32 complex).
Error launch_rows_wave(int n_px, const ImageArgs &a, int l0, int cnt, cudaStream_t st);

// Pass 2 as a dense real GEMM on the tensor cores (blink_dftgemm.cu).
// mode: 1 BF16, 2 BF16 x3 (split-precision), 3 FP16, 4 FP16 x3.
bool dftgemm_supported(int n_px, int r_alloc, int mode);
size_t dftgemm_scratch_per_layer(int n_px, int r_alloc);
// Layer-independent part of that scratch (DFT tables of both passes).
size_t dftgemm_scratch_fixed(int n_px, int r_alloc, int kmax);
Error launch_dftgemm_group(int n_px, int mode, const ImageArgs &a, cudaStream_t st);

// Whether the column pass of size n_px (FFT path) transforms the adjoint's
// columns as it stores them (else they come from the stored images).
bool adjoint_fusable(int n_px);
// Slots of sq_part one layer of size n_px can use (its column items).
int sq_slots(int n_px);
// out[l] = sum over s < stride of part[l * stride + s], in slot order.
Error launch_sq_totals(const double *part, int stride, int n_layers, double *out, cudaStream_t st);

// Adjoint of the image path: resid (float [N][N] at out_off) -> dvis
// (complex64 at vis_off).  Needs degrid_scratch_per_layer() bytes per layer.
size_t degrid_scratch_per_layer(int n_px, int r_alloc);
Error launch_degrid_group(int n_px, const ImageArgs &a, const float *resid, float2 *dvis, cudaStream_t st);
// The two halves of that adjoint with the column transforms kept in between
// (slots of r_alloc rows of N complex per layer of the group).
Error launch_degrid_cols_group(int n_px, const ImageArgs &a, const float *resid, float2 *out, cudaStream_t st);
Error launch_degrid_rows_group(int n_px, const ImageArgs &a, const float2 *in, float2 *dvis, cudaStream_t st);

// Antenna gains (blink_gains.cu): vis = g_i conj(g_j) model per layer, and
// the per-antenna gradient accumulated over all layers.
// out[r][b] = g_i conj(g_j) of gain row r (gains + r * stride), r < rows.
Error launch_gain_products(const float2 *gains, int64_t stride, int rows, int n_ant, int64_t nb, float2 *out,
                           cudaStream_t st);
Error launch_apply_gains(const float2 *model, const float2 *gains, const int64_t *vis_off, int n_layers, int n_ant,
                         int64_t nb, float2 *vis, cudaStream_t st);
// Device scratch of launch_gain_grad (per-tile and per-row FP64 partials).
size_t gain_grad_scratch_bytes(int n_layers, int n_ant);
Error launch_gain_grad(const float2 *dvis, const float2 *model, const float2 *gains, const int64_t *vis_off,
                       int n_layers, int n_ant, float2 *dgains, void *scratch, cudaStream_t st);

}  // namespace blink
