// rt_fit_gains_noalloc: the per-camera gain fit of one frame set without any
// allocation, for callers that cannot call cudaMalloc (a process whose device
// memory belongs to another allocator or is reserved up front, a plug-in that
// must not grow the device footprint): the band statistics, the work list and
// the seam tables live in one file-scope device array.
//
// The array is shared by every call in the process: calls that overlap on
// the GPU (different streams, or the same array used before a previous call
// finished) race on it.  Its contents persist between calls; the statistics
// part is cleared at the start of every call.  Nothing is copied from host
// memory: the work list and the seam tables are written into the array by a
// small set-up kernel from its by-value parameter block.
#include <atomic>
#include <cstring>

#include "rt_internal.cuh"
#include "pixel.cuh"

using namespace rt;

namespace {

constexpr int kNaCams = 16;        // cameras
constexpr int kNaBlocks = 4;       // vertical blocks
constexpr int kNaStrip = 32;       // band width
constexpr int kNaRows = 2160;      // rows per camera
constexpr int kNaItemRows = 64;    // rows of one band work item
constexpr int kNaItems = kNaCams * 2 * (kNaBlocks + kNaRows / kNaItemRows + 1);

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t kNb = (size_t)kNaCams * 2 * kNaBlocks;            // (camera, side, block) slots
constexpr size_t kOffHist = 0;                                       // u32 [slots][3][256] + n [slots][3]
constexpr size_t kHistBytes = (kNb * 768 + kNb * 3) * 4;
constexpr size_t kOffSum = (kOffHist + kHistBytes + 255) / 256 * 256; // u64 sums [slots][3], sumsq [slots][3]
constexpr size_t kSumBytes = kNb * 3 * 2 * 8;
constexpr size_t kOffLuma = (kOffSum + kSumBytes + 255) / 256 * 256;  // u8 [cams][2][rows][strip]
constexpr size_t kLumaBytes = (size_t)kNaCams * 2 * kNaRows * kNaStrip;
constexpr size_t kOffItems = (kOffLuma + kLumaBytes + 255) / 256 * 256;
constexpr size_t kItemsBytes = (size_t)kNaItems * sizeof(StripItem);
constexpr size_t kOffTables = (kOffItems + kItemsBytes + 255) / 256 * 256;   // int32 tables
constexpr int kTableInts = (kNaCams + 1) + kNaCams * 4;
constexpr size_t kScratchBytes = (kOffTables + kTableInts * 4 + 255) / 256 * 256;

static_assert(kScratchBytes == 2632704, "the documented size of the scratch array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of the array, per device (looked up once, on first use;
// concurrent first calls store the same value)
constexpr int kMaxDevices = 64;
std::atomic<void *> g_scratch_addr[kMaxDevices];

rt_status scratch_for_current_device(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RT_ERR_CUDA;
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RT_ERR_CUDA;
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return RT_OK;
}

// What the set-up kernel needs to write the band work list and the seam
// tables (by value, a few hundred bytes).
struct NaSetup {
    int32_t K, B;
    int32_t H[kNaCams];
    int32_t tables[kTableInts];
};

// Work items in the order the host counts them: camera, side, block, then
// kNaItemRows-row pieces of the block; then the seam tables.
__global__ void noalloc_setup_kernel(const NaSetup a, StripItem *__restrict__ items, int32_t *__restrict__ tab)
{
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < a.K; ++k)
            for (int side = 0; side < 2; ++side)
                for (int j = 0; j < a.B; ++j) {
                    const int H = a.H[k];
                    const int r0 = (int)(((long long)j * H) / a.B), r1 = (int)(((long long)(j + 1) * H) / a.B);
                    for (int r = r0; r < r1; r += kNaItemRows) {
                        StripItem it;
                        it.cam = (int16_t)k; it.side = (int16_t)side; it.block = (int16_t)j; it.pad = 0;
                        it.row0 = r; it.row1 = r + kNaItemRows < r1 ? r + kNaItemRows : r1;
                        items[n++] = it;
                    }
                }
    }
    for (int i = threadIdx.x; i < kTableInts; i += blockDim.x) tab[i] = a.tables[i];
}

}  // namespace

extern "C" rt_status rt_fit_gains_noalloc(const rt_camera_desc *cams, int32_t num_cameras,
                                          const void *const *y_planes, const void *const *uv_planes,
                                          int32_t strip_width, int32_t num_blocks, int32_t topology,
                                          double *maps_dev, int32_t *q16_dev, void *cuda_stream)
{
    const int K = num_cameras, B = num_blocks, S = strip_width;
    if (!cams || !y_planes || !maps_dev || !q16_dev) return RT_ERR_INVALID;
    if (K < 1 || K > kNaCams || B < 1 || B > kNaBlocks || S < 16 || S > kNaStrip || S % 16) return RT_ERR_INVALID;
    if (topology != RT_LINEAR && topology != RT_RING) return RT_ERR_INVALID;
    if (((uintptr_t)maps_dev & 7) || ((uintptr_t)q16_dev & 3)) return RT_ERR_INVALID;
    for (int k = 0; k < K; ++k) {
        const rt_camera_desc &c = cams[k];
        const int bpp = c.format == RT_MONO16 ? 2 : 1;
        if (c.format != RT_NV12 && c.format != RT_MONO16) return RT_ERR_INVALID;
        if (c.width < 2 * S || c.width % 2 || c.height < 2 || c.height % 2 || c.height > kNaRows || c.height < B)
            return RT_ERR_INVALID;
        if (c.y_pitch % 16 || c.y_pitch < (c.width * bpp + 15) / 16 * 16) return RT_ERR_INVALID;
        if (c.format == RT_MONO16 && (c.bit_depth < 8 || c.bit_depth > 16)) return RT_ERR_INVALID;
        if (!y_planes[k] || ((uintptr_t)y_planes[k] & 15)) return RT_ERR_INVALID;
        if (c.format == RT_NV12) {
            if (c.uv_pitch % 16 || c.uv_pitch < (c.width + 15) / 16 * 16) return RT_ERR_INVALID;
            if (!uv_planes || !uv_planes[k] || ((uintptr_t)uv_planes[k] & 15)) return RT_ERR_INVALID;
        }
        if (c.group < 0) return RT_ERR_INVALID;
        for (int q = 0; q < k; ++q)
            if (cams[q].group == c.group && cams[q].position == c.position) return RT_ERR_INVALID;
    }
    void *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != RT_OK) return RT_ERR_CUDA;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // geometry of this frame set (kernel parameters)
    ArrayGeom g;
    memset(&g, 0, sizeof g);
    g.K = K; g.B = B; g.fit_mode = RT_FIT_GLOBAL; g.matrix = RT_BT709;
    g.conv = conv_consts(RT_BT709);
    int Hmax = 0;
    for (int k = 0; k < K; ++k) {
        CamGeom &cg = g.cam[k];
        cg.y = static_cast<const uint8_t *>(y_planes[k]);
        cg.uv = cams[k].format == RT_NV12 ? static_cast<const uint8_t *>(uv_planes[k]) : nullptr;
        cg.W = cams[k].width; cg.H = cams[k].height;
        cg.y_pitch = cams[k].y_pitch; cg.uv_pitch = cams[k].uv_pitch;
        cg.fmt = cams[k].format; cg.shift = cams[k].format == RT_MONO16 ? cams[k].bit_depth - 8 : 0;
        cg.nblk = B;
        if (cg.H > Hmax) Hmax = cg.H;
    }
    // band work items (counted here, written by the set-up kernel) and seam tables
    NaSetup su;
    memset(&su, 0, sizeof su);
    su.K = K; su.B = B;
    int n_items = 0;
    for (int k = 0; k < K; ++k) {
        su.H[k] = cams[k].height;
        for (int j = 0; j < B; ++j) {
            const int H = cams[k].height;
            const int r0 = (int)(((long long)j * H) / B), r1 = (int)(((long long)(j + 1) * H) / B);
            n_items += 2 * ((r1 - r0 + kNaItemRows - 1) / kNaItemRows);
        }
    }
    int32_t *tables = su.tables;
    int32_t *gs = tables, *gm = tables + (kNaCams + 1), *ln = gm + kNaCams, *rn = ln + kNaCams, *hh = rn + kNaCams;
    int n_groups = 0, n_members = 0;
    gs[0] = 0;
    for (int k = 0; k < K; ++k) { ln[k] = -1; rn[k] = -1; hh[k] = cams[k].height; }
    bool done[kNaCams] = {};
    for (int start = 0; start < K; ++start) {
        if (done[start]) continue;
        const int grp = cams[start].group;
        int m[kNaCams], nm = 0;
        for (int k = 0; k < K; ++k)
            if (cams[k].group == grp) { m[nm++] = k; done[k] = true; }
        for (int a = 1; a < nm; ++a)      // order by position
            for (int b = a; b > 0 && cams[m[b]].position < cams[m[b - 1]].position; --b) {
                const int tmp = m[b]; m[b] = m[b - 1]; m[b - 1] = tmp;
            }
        for (int i = 0; i < nm; ++i) {
            gm[n_members++] = m[i];
            if (i + 1 < nm) { rn[m[i]] = m[i + 1]; ln[m[i + 1]] = m[i]; }
        }
        if (topology == RT_RING && nm >= 2) { rn[m[nm - 1]] = m[0]; ln[m[0]] = m[nm - 1]; }
        gs[++n_groups] = n_members;
    }
    StripItem *d_items = reinterpret_cast<StripItem *>(base + kOffItems);
    int32_t *d_tab = reinterpret_cast<int32_t *>(base + kOffTables);
    noalloc_setup_kernel<<<1, 128, 0, st>>>(su, d_items, d_tab);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    // statistics start at zero
    if (cudaMemsetAsync(base + kOffHist, 0, kHistBytes, st) != cudaSuccess ||
        cudaMemsetAsync(base + kOffSum, 0, kSumBytes, st) != cudaSuccess)
        return RT_ERR_CUDA;

    const size_t nb = (size_t)K * 2 * B;
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + kOffHist);
    unsigned long long *sum = reinterpret_cast<unsigned long long *>(base + kOffSum);
    PassAArgs pa{};
    pa.items = d_items; pa.n_items = n_items; pa.S = S; pa.T = 255; pa.first = 1;
    pa.prev_luma = nullptr; pa.cur_luma = base + kOffLuma;
    pa.luma_cam_stride = 2 * Hmax * S;
    pa.hist = hist; pa.n = hist + nb * 768; pa.sum = sum; pa.sumsq = sum + nb * 3;
    pa.clear_u32 = nullptr; pa.clear_u32_n = 0; pa.clear_u64 = nullptr; pa.clear_u64_n = 0;
    if (launch_pass_a(g, pa, 64, st) != cudaSuccess) return RT_ERR_CUDA;

    SolveArgs sa{};
    sa.n = pa.n; sa.sum = pa.sum; sa.sumsq = pa.sumsq;
    sa.maps_new = maps_dev; sa.E = maps_dev; sa.q16 = q16_dev;   // first estimate: E = E_new
    sa.K = K; sa.B = B; sa.S = S; sa.fit_mode = RT_FIT_GLOBAL; sa.min_valid = 64; sa.first = 1;
    sa.alpha = 0.05; sa.lambda = 1e-6; sa.gmin = 0.25; sa.gmax = 4.0;
    sa.n_groups = n_groups; sa.group_start = d_tab; sa.group_members = d_tab + (kNaCams + 1);
    sa.left_nbr = sa.group_members + kNaCams; sa.right_nbr = sa.left_nbr + kNaCams; sa.cam_H = sa.right_nbr + kNaCams;
    fill_solve_topo(sa.topo, K, n_groups, gs, gm, rn, hh);
    if (launch_solve(sa, st) != cudaSuccess) return RT_ERR_CUDA;
    return RT_OK;
}
