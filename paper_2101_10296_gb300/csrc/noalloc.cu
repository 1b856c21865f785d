// qaoa_energy_noalloc: the energy evaluation of qaoa_energy, for callers that
// must not allocate device memory while they run -- for instance code running
// inside a custom allocator's callback, under a memory-budget manager that
// forbids new allocations, or in a process whose allocator is owned by
// another runtime.  All of its temporary memory (the phase tables and the
// state blocks of cones on the large-state path) comes from one file-scope
// device array of fixed size instead of cudaMallocAsync.  Nothing is
// allocated by this call; the plan's own device copy must already exist
// (qaoa_plan_upload, a set-up step that does allocate).  The array itself
// takes device memory when the CUDA module holding it is loaded, which with
// lazy module loading happens at the first use of its symbol: the upload
// makes that first use (noalloc_prepare), so the array's memory is committed
// during set-up and not inside a qaoa_energy_noalloc call.
#include <mutex>
#include <string>

#include "big.cuh"
#include "device.cuh"
#include "devplan.cuh"
#include "host.hpp"

using namespace qaoa;

namespace {

constexpr size_t kNoAllocBytes = size_t(QAOA_NOALLOC_SCRATCH_MB) << 20;

// The scratch every qaoa_energy_noalloc call shares.  Each device that loads
// the library holds one copy until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the array on the current device, looked up once per
// device (host code cannot use the symbol's name as a device address).
int scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
            return QAOA_E_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return QAOA_OK;
}

}  // namespace

namespace qaoa {
// Looks up the array's address on the current device (loading its module, the
// one allocation the array ever makes).  Called by qaoa_plan_upload; a failure
// there is not fatal, since qaoa_energy_noalloc repeats the lookup and reports
// it.
int noalloc_prepare() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QAOA_E_CUDA;
    unsigned char *p = nullptr;
    return scratch_address(dev, &p);
}
}  // namespace qaoa

extern "C" int qaoa_energy_noalloc(const qaoa_plan *plan, int64_t n_points, const double *params_dev,
                                   double *energy_dev, double *terms_dev, qaoa_stream_t stream) {
    if (!plan || n_points < 1 || !params_dev || !energy_dev) {
        set_error("need a plan, n_points >= 1, params and energy");
        return QAOA_E_INVALID;
    }
    if (!plan->dev) {
        set_error("qaoa_energy_noalloc needs a plan already copied to the device (qaoa_plan_upload)");
        return QAOA_E_INVALID;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return QAOA_E_CUDA;
    }
    if (dev != plan->dev->device || dev < 0 || dev >= kMaxDevices) {
        set_error("the plan lives on device " + std::to_string(plan->dev->device) + ", current device is " +
                  std::to_string(dev));
        return QAOA_E_INVALID;
    }
    const qaoa_device_plan *d = plan->dev;
    const int32_t G = plan->n_graphs, p = plan->p;
    const size_t GP = size_t(G) * size_t(n_points);
    // carve the static array; refuse before launching anything if it is too small
    const size_t lut_b = align256(GP * p * d->cmax1 * sizeof(float2));
    const size_t mix_b = align256(GP * p * sizeof(float2));
    const size_t kpow_b = align256(GP * p * kKpow * sizeof(float));
    const size_t cs_b = d->big.empty() ? 0 : align256(GP * p * sizeof(float4));
    const size_t tables = lut_b + mix_b + kpow_b + cs_b;
    size_t largest_block = 0;
    for (const BigShape &bs : d->big)
        largest_block = std::max(largest_block, (size_t(1) << bs.n_in) * sizeof(float2));
    if (tables + largest_block > kNoAllocBytes) {
        set_error("qaoa_energy_noalloc: " + std::to_string(n_points) + " points need " +
                  std::to_string((tables + largest_block + (1 << 20) - 1) >> 20) +
                  " MiB of scratch, more than its fixed " + std::to_string(kNoAllocBytes >> 20) +
                  " MiB (use qaoa_energy, or fewer points per call)");
        return QAOA_E_INVALID;
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc != QAOA_OK) return rc;
    float2 *lut = reinterpret_cast<float2 *>(base);
    float2 *mix = reinterpret_cast<float2 *>(base + lut_b);
    float *kpow = reinterpret_cast<float *>(base + lut_b + mix_b);
    float4 *cs = reinterpret_cast<float4 *>(base + lut_b + mix_b + kpow_b);
    unsigned char *blocks = base + tables;
    const size_t block_room = kNoAllocBytes - tables;
    cudaStream_t s = (cudaStream_t)stream;

    // phase tables and output initialisation (every table entry and output is
    // written before it is read, so nothing in the array needs clearing)
    PrepArgs pa;
    pa.params = params_dev;
    pa.G = G;
    pa.p = p;
    pa.cmax1 = d->cmax1;
    pa.P = n_points;
    pa.half_edges = d->half_edges;
    pa.lut = lut;
    pa.mix = mix;
    pa.kpow = kpow;
    pa.energy = energy_dev;
    pa.grad = nullptr;
    pa.terms = terms_dev;
    pa.n_reps = d->n_cones;
    e = launch_prep(pa, s);
    // register-resident cones: the depth-1 kernel where the plan has its list
    // (p = 1, no per-cone terms asked for), else the general register kernel
    if (e == cudaSuccess && p == 1 && d->reg_p1.warps > 0 && terms_dev == nullptr) {
        RegLaunch L;
        L.work = reg_work(d, d->reg_p1);
        L.n_points = n_points;
        L.p = 1;
        const int64_t row = int64_t(d->cmax1 + 1) * int64_t(sizeof(float2));
        const int64_t fixed = int64_t(reg_p1_smem_bytes(0, d->cmax1, false)) / (kRegBlock / 32);
        const int64_t fit = (int64_t(kRegMaxSmem) / (kRegBlock / 32) - fixed) / row;
        L.jpt = int32_t(std::min<int64_t>(std::min<int64_t>(8, std::max<int64_t>(1, fit)), n_points));
        L.cmax1 = d->cmax1;
        L.lut = lut;
        L.mix = mix;
        L.kpow = kpow;
        L.energy = energy_dev;
        L.grad = nullptr;
        L.terms = nullptr;
        L.status = d->status;
        const size_t smem = reg_p1_smem_bytes(L.jpt, d->cmax1, false);
        const int64_t tasks = L.work.warps * ((n_points + L.jpt - 1) / L.jpt);
        const int64_t grid = std::min<int64_t>(reg_p1_grid(false, smem), (tasks + 3) / 4);
        e = launch_reg_p1(L, false, int(std::max<int64_t>(grid, 1)), s);
    } else if (e == cudaSuccess && d->reg_e.warps > 0) {
        RegLaunch L;
        L.work = reg_work(d, d->reg_e);
        L.n_points = n_points;
        L.p = p;
        const int64_t row_bytes = int64_t(p) * ((d->cmax1 + 1) * int64_t(sizeof(float2)) + kRegKpow * int64_t(sizeof(float)));
        L.jpt = int32_t(std::min<int64_t>(std::min<int64_t>(8, std::max<int64_t>(1, 6144 / row_bytes)), n_points));
        L.cmax1 = d->cmax1;
        L.lut = lut;
        L.mix = mix;
        L.kpow = kpow;
        L.energy = energy_dev;
        L.grad = nullptr;
        L.terms = terms_dev;
        L.status = d->status;
        const bool wide = d->cmax1 - 1 > 32;
        const size_t smem = reg_smem_bytes(L.jpt, p, d->cmax1, false);
        const int64_t tasks = d->reg_e.warps * ((n_points + L.jpt - 1) / L.jpt);
        const int64_t grid = std::min<int64_t>(reg_energy_grid(wide, smem), (tasks + 3) / 4);
        e = launch_reg_energy(L, wide, int(std::max<int64_t>(grid, 1)), s);
    }
    // large-state cones: waves sized to the room left in the array
    if (e == cudaSuccess && !d->big.empty()) {
        e = launch_big_prep(params_dev, int64_t(GP), p, cs, nullptr, s);
        const int grid = big_grid(false);
        int64_t launches = 0;
        for (const BigShape &bs : d->big) {
            if (e != cudaSuccess) break;
            const size_t block_bytes = (size_t(1) << bs.n_in) * sizeof(float2);
            const int64_t items = bs.ystart.back() * n_points;
            const int64_t wave = std::max<int64_t>(1, std::min<int64_t>(items, int64_t(block_room / block_bytes)));
            BigLaunch B{};
            B.cones = d->cones;
            B.cone_ids = bs.d_cones;
            B.ystart = bs.d_ystart;
            B.n_shape = int32_t(bs.cones.size());
            B.n_in = bs.n_in;
            B.P = n_points;
            B.p = p;
            B.cmax1 = d->cmax1;
            B.lut = lut;
            B.cs = cs;
            B.fa = nullptr;
            B.mix = mix;
            B.kpow = kpow;
            B.psi = reinterpret_cast<float2 *>(blocks);
            B.shell = d->shell;
            B.lam = nullptr;
            B.energy = energy_dev;
            B.grad = nullptr;
            B.terms = terms_dev;
            B.status = d->status;
            for (int64_t i0 = 0; i0 < items && e == cudaSuccess; i0 += wave) {
                B.item0 = i0;
                B.n_items = std::min(wave, items - i0);
                if (bs.split_e) {
                    e = launch_split_wave(B, false, d->chunk_window, launches, s);
                    continue;
                }
                for (const BigPass &ps : bs.fwd) {
                    B.pass = ps;
                    e = launch_big_pass(B, false, grid, s);
                    if (e != cudaSuccess) break;
                }
            }
        }
    }
    if (e != cudaSuccess) {
        set_error(std::string("qaoa_energy_noalloc launch: ") + cudaGetErrorString(e));
        return QAOA_E_CUDA;
    }
    return QAOA_OK;
}
