// tpc_noalloc.cu -- neighbour links of one event without any allocation.
//
// Some callers cannot allocate device memory: code that runs inside a
// host-side framework owning the device allocator (an allocation there
// would bypass its accounting or deadlock against its pool), code that runs
// with a hard memory budget where a cudaMalloc could fail at an arbitrary
// moment, and callers that must not trigger the device synchronisation a
// cudaMalloc/cudaFree can imply.  For them tpc_track_links_noalloc runs the
// binning and neighbour-finding kernels of the tracker on scratch memory that
// is a file-scope static device array of this library: it is created when
// the library is loaded on a device and held by every device that loads the
// library until the process exits, so it is kept modest (kNaBytes).
//
// The static array is named directly only in device code; host code needs
// its device address, which cudaGetSymbolAddress returns once per device,
// with that device current, on the first call made on the device.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/tpctrack.h"
#include "tpc_internal.cuh"

namespace tpc {
namespace {

constexpr long long kNaMaxClusters = 131072;  // clusters per call
constexpr int kNaMaxSectors = 36;             // sectors per call
constexpr int kNaMaxDevices = 64;

// Layout of the scratch array (every size a multiple of 256 bytes).
constexpr size_t up256(size_t v) { return (v + 255) / 256 * 256; }
constexpr long long kNaRS = (long long)kNaMaxSectors * kMaxRows;
constexpr long long kNaBins = kNaMaxClusters * kBinsPerHitX2 / 2 + 2 * kNaRS + 16;
constexpr long long kNaRowTiles = kNaRS / kRowTile + 2;
constexpr long long kNaHitTiles = kNaMaxClusters / kHitTile + 2;
constexpr size_t kNaDesc = up256(sizeof(EventDesc) + 2 * sizeof(long long) +
                                 sizeof(int) * kNaMaxSectors + sizeof(float) * kMaxRows);
constexpr size_t kNaZero = up256(up256(sizeof(Counters)) + 4 * (kNaRS * kCntPad + 2 * kNaMaxSectors + 4) +
                                 8 * (kNaRowTiles + kNaHitTiles + kNaMaxSectors) + 1024);
constexpr size_t kNaBytes =
    kNaDesc + kNaZero + up256(4 * (kNaRS + 1)) + up256(4 * kNaRS) + up256(sizeof(RowGrid) * kNaRS) +
    up256(4 * kNaBins) + 9 * up256(4 * kNaMaxClusters) /* tmp rec (4), rank, hyz (2), hcid, hrow */ +
    2 * up256(4 * kNaMaxClusters) /* up dn */ + 2 * up256(4 * kNaMaxClusters) /* upc dnc */ +
    up256(4 * kNaMaxClusters) /* upg */ + up256(8 * kNaMaxClusters) /* weight */ +
    up256(4 * kNaMaxClusters) /* starts */ + up256(4 * kNaMaxClusters) /* crowded */;

// The scratch: shared by every call on a device and holding the last call's
// contents; whatever must start at zero is cleared at the start of a call.
static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {nullptr};
Schedule g_na_sched[kNaMaxDevices];

// Links of every sorted hit as input cluster ids (or -1).
__global__ void k_links_by_cid(Launch L, int32_t* up_cid, int32_t* dn_cid)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n = L.row_off[L.RS];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int hr = L.hrow[i];
        const int g = (hr >> 8) * L.R + (hr & 255);
        const int u = L.up[i], d = L.dn[i];
        const int c = L.hcid[i];
        up_cid[c] = u >= 0 ? L.hcid[L.row_off[g + 1] + u] : -1;
        dn_cid[c] = d >= 0 ? L.hcid[L.row_off[g - 1] + d] : -1;
    }
}

}  // namespace
}  // namespace tpc

using namespace tpc;

extern "C" int tpc_track_links_noalloc(const tpc_clusters* ev, const tpc_geometry* g,
                                       const tpc_track_params* P, int32_t* up_cid,
                                       int32_t* dn_cid, void* cuda_stream)
{
    if (!ev || !g || !P || !up_cid || !dn_cid) return TPC_EINVAL;
    if (!ev->on_device) return TPC_EINVAL;
    if (ev->n < 0 || ev->n > kNaMaxClusters) return TPC_EINVAL;  // beyond the static scratch
    if (ev->n > 0 && (!ev->y || !ev->z || !ev->row || !ev->sector)) return TPC_EINVAL;
    if (!g->row_x || g->n_rows < 3 || g->n_rows > kMaxRows) return TPC_EINVAL;
    for (int r = 1; r < g->n_rows; ++r)
        if (!(g->row_x[r] > g->row_x[r - 1])) return TPC_EINVAL;
    const int n_sec = g->n_sectors_phi * (g->split_z ? 2 : 1);
    if (g->n_sectors_phi < 1 || n_sec > kNaMaxSectors) return TPC_EINVAL;
    if (!(g->half_angle_rad > 0.0f && g->half_angle_rad < 1.5f) || !(g->z_max > 0.0f))
        return TPC_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return TPC_ECUDA;
    // once per device, with the device current: device address of the scratch
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return TPC_ECUDA;
            }
            prepare_kernels(&g_na_sched[dev]);
            g_na_ptr[dev] = p;
        }
        base = (unsigned char*)g_na_ptr[dev];
    }
    const Schedule& sched = g_na_sched[dev];
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += up256(bytes);
        return p;
    };
    const long long n = ev->n;
    const int R = g->n_rows;
    Launch L;
    std::memset(&L, 0, sizeof(L));
    L.n_total = n;
    L.n_events = 1;
    L.R = R;
    L.S = n_sec;
    L.RS = n_sec * R;
    L.n_sectors_phi = g->n_sectors_phi;
    L.split_z = g->split_z ? 1 : 0;
    L.t_cap = (int)kNaMaxClusters;
    L.tan_half = tanf(g->half_angle_rad);
    L.z_max = g->z_max;
    L.slope_win_y = P->slope_win_y;
    L.slope_win_z = P->slope_win_z;
    L.d_max = P->d_max;
    // descriptors: one event, its cluster offsets, sector -> event, row radii
    unsigned char* desc = take(kNaDesc);
    struct {
        EventDesc e;
        long long off[2];
        int sec_event[kNaMaxSectors];
        float xr[kMaxRows];
    } h;
    std::memset(&h, 0, sizeof(h));
    h.e.y = ev->y;
    h.e.z = ev->z;
    h.e.row = ev->row;
    h.e.sec = ev->sector;
    h.e.n = n;
    h.e.cl_off = 0;
    h.e.sec_base = 0;
    h.e.n_sec = n_sec;
    h.off[0] = 0;
    h.off[1] = n;
    for (int r = 0; r < R; ++r) h.xr[r] = g->row_x[r];
    L.ev = (EventDesc*)desc;
    L.ev_off = (long long*)(desc + offsetof(decltype(h), off));
    L.sec_event = (int*)(desc + offsetof(decltype(h), sec_event));
    L.xr = (const float*)(desc + offsetof(decltype(h), xr));
    // zero region: counters, row counts and fill counters, look-back states
    unsigned char* zero = take(kNaZero);
    {
        size_t zo = 0;
        auto z = [&](size_t bytes) {
            zo = (zo + 15) / 16 * 16;
            unsigned char* p = zero + zo;
            zo += bytes;
            return p;
        };
        L.cnt = (Counters*)z(sizeof(Counters));
        L.row_cnt = (int*)z(4 * (size_t)L.RS * kCntPad);
        L.ev_invalid = (int*)z(4);
        L.sec_first = (int*)z(4 * (size_t)n_sec);
        L.sec_end = (int*)z(4 * (size_t)n_sec);
        L.n_row_tiles = (int)((L.RS + kRowTile - 1) / kRowTile);
        L.n_hit_tiles = (int)((n + kHitTile - 1) / kHitTile);
        if (L.n_hit_tiles < 1) L.n_hit_tiles = 1;
        L.tile_state = (unsigned long long*)z(8 * ((size_t)L.n_row_tiles + L.n_hit_tiles + n_sec));
        if (cudaMemsetAsync(zero, 0, zo, st) != cudaSuccess) return TPC_ECUDA;
    }
    L.row_off = (int*)take(4 * (kNaRS + 1));
    L.big_rows = (int*)take(4 * kNaRS);
    L.grid = (RowGrid*)take(sizeof(RowGrid) * kNaRS);
    L.bin_start = (int*)take(4 * kNaBins);
    L.tmp_rec = (float4*)take(16 * kNaMaxClusters);
    L.rank = (int*)take(4 * kNaMaxClusters);
    L.hyz = (float2*)take(8 * kNaMaxClusters);
    L.hcid = (int*)take(4 * kNaMaxClusters);
    L.hrow = (int*)take(4 * kNaMaxClusters);
    L.up = (int16_t*)take(4 * kNaMaxClusters);
    L.dn = (int16_t*)take(4 * kNaMaxClusters);
    L.upc = (int16_t*)take(4 * kNaMaxClusters);
    L.dnc = (int16_t*)take(4 * kNaMaxClusters);
    L.upg = (int*)take(4 * kNaMaxClusters);
    L.weight = (unsigned long long*)take(8 * kNaMaxClusters);
    L.starts = (int*)take(4 * kNaMaxClusters);
    L.crowded = (int*)take(4 * kNaMaxClusters);
    if (off > kNaBytes) return TPC_EINVAL;  // layout and size disagree (cannot happen)
    if (cudaMemcpyAsync(desc, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return TPC_ECUDA;
    launch_binning(L, sched, st, nullptr);
    launch_finder(L, sched, st, nullptr);
    const int blocks = (int)((n + 255) / 256) > 0 ? (int)((n + 255) / 256) : 1;
    k_links_by_cid<<<blocks < 1184 ? blocks : 1184, 256, 0, st>>>(L, up_cid, dn_cid);
    // a launch error is left pending for the caller (an error already pending
    // on this thread from earlier work is reported the same way)
    if (cudaPeekAtLastError() != cudaSuccess) return TPC_ECUDA;
    Counters c;
    if (cudaMemcpyAsync(&c, L.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return TPC_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TPC_ECUDA;
    if (c.n_invalid) return TPC_EINVAL;
    if (c.ovf_row) return TPC_ECAPACITY;
    if (c.timeout) return TPC_ETIMEOUT;
    return TPC_OK;
}
