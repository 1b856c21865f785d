// C-ABI device entry points: plan upload, energy / gradient launches,
// cut tables, device status.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "big.cuh"
#include "device.cuh"
#include "devplan.cuh"
#include "host.hpp"

using namespace qaoa;

namespace qaoa {
int noalloc_prepare();  // noalloc.cu
}

namespace {

int cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QAOA_E_OOM : QAOA_E_CUDA;
}

void free_work(DevWork &w) {
    cudaFree(w.slot_cone);
    cudaFree(w.warp_graph);
    cudaFree(w.rec_hi);
    cudaFree(w.rec_wk);
    cudaFree(w.rec_cw);
    w = DevWork{};
}

// Shell word and multiplicity of block beta of a cone, decoded from the shell
// table exactly as the kernels' shell_block does (the same float products in
// the same order).
uint64_t host_shell_block(const DevCone &C, const std::vector<uint64_t> &tab, uint32_t beta, float &mult) {
    if (C.n_cls < 0) {
        if (int64_t(beta) >= C.n_blocks) {
            mult = 0.f;
            return 0;
        }
        const uint64_t *e = tab.data() + C.cls_off + 2 * size_t(beta);
        const uint32_t bits = uint32_t(e[1]);
        std::memcpy(&mult, &bits, sizeof mult);
        return e[0];
    }
    const uint64_t *t = tab.data() + C.cls_off;
    uint64_t m = 0;
    float w = 1.f;
    for (int c = 0; c < C.n_cls; ++c) {
        const uint32_t sz = uint32_t(t[0]);
        const uint32_t q = beta / (sz + 1);
        const uint32_t nc = beta - q * (sz + 1);
        beta = q;
        m ^= t[1 + nc];
        const uint32_t bits = uint32_t(t[2 + sz + nc]);
        float f;
        std::memcpy(&f, &bits, sizeof f);
        w *= f;
        t += 2 * sz + 3;
    }
    mult = w;
    return m;
}

// Builds the slot list for R register qubits over the given plan indices:
// cones sorted by (G_c = 2^max(n_in - R, 0) descending, graph, plan order)
// and packed back to back, T_c slots each (a multiple of G_c, so every cone
// starts at a multiple of its own G_c and its lane-qubit groups never
// straddle a cone boundary); a new graph starts on a fresh warp.  Then the
// slot records (see RegWork): for slot s of cone c at offset t = s - start_c
// the thread holds inner qubits R..n_in-1 in the low bits of t and block
// group t >> max(n_in - R, 0); register bits [2, nr) are inner qubits (nr =
// min(n_in, R)) and bits [nr, R) pick one of 2^(R - nr) blocks of the group.
int build_work(const std::vector<DevCone> &hc, const std::vector<uint64_t> &shell_tab,
               const std::vector<int32_t> &idx, int R, bool wide, DevWork &w) {
    std::vector<int32_t> order(idx);
    auto G = [&](int32_t i) { return int64_t(1) << std::max(hc[i].n_in - R, 0); };
    auto T = [&](int32_t i) {
        const int sb = std::max(R - hc[i].n_in, 0);
        return ((hc[i].n_blocks + (int64_t(1) << sb) - 1) >> sb) * G(i);
    };
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (G(a) != G(b)) return G(a) > G(b);
        return hc[a].graph < hc[b].graph;
    });
    std::vector<int64_t> start(order.size() + 1, 0);
    int64_t pos = 0;
    for (size_t i = 0; i < order.size(); ++i) {
        if (i > 0 && hc[order[i]].graph != hc[order[i - 1]].graph) pos = (pos + 31) / 32 * 32;
        start[i] = pos;
        pos += T(order[i]);
    }
    pos = (pos + 31) / 32 * 32;
    start[order.size()] = pos;
    const int64_t slots = pos;
    const int64_t warps = slots / 32;
    w.slots = slots;
    w.warps = warps;
    w.n = int32_t(order.size());
    if (order.empty()) return QAOA_OK;
    const int S = 1 << (R - 2);
    std::vector<int32_t> wgraph(size_t(warps), 0);
    std::vector<int32_t> scone(size_t(slots), 0);
    std::vector<uint64_t> hi64(size_t(S) * size_t(slots), 0);
    std::vector<float> wk(size_t(S) * size_t(slots), 0.f);
    size_t ci = 0;
    for (int64_t sl = 0; sl < slots; ++sl) {
        // the cone owning the slot: the last one starting at or before it
        while (ci + 1 < order.size() && start[ci + 1] <= sl) ++ci;
        const DevCone &C = hc[size_t(order[ci])];
        const bool active = sl < start[ci] + T(order[ci]);
        scone[size_t(sl)] = order[ci] | (active ? 0 : int32_t(0x80000000u));
        if (sl % 32 == 0) wgraph[size_t(sl / 32)] = C.graph;
        const int64_t t = active ? sl - start[ci] : 0;  // padding: the cone's first slot, weight 0
        const int n_in = C.n_in;
        const int nr = std::min(n_in, R);
        const int gb = std::max(n_in - R, 0);
        const int sb = R - nr;
        const int inner_bits = nr - 2;
        uint64_t base = 0;
        for (int q = R; q < n_in; ++q)
            if ((t >> (q - R)) & 1) base ^= C.col[q];
        const uint32_t group = uint32_t(t >> gb);
        uint64_t shell = 0;
        float mult = 0.f;
        for (int k = 0; k < S; ++k) {
            if ((k & ((1 << inner_bits) - 1)) == 0) {
                const uint32_t beta = (group << sb) + uint32_t(k >> inner_bits);
                shell = host_shell_block(C, shell_tab, beta, mult);
                if (int64_t(beta) >= C.n_blocks) mult = 0.f;
            }
            uint64_t v = base ^ shell;
            for (int b = 0; b < R - 2; ++b)
                if (((k >> b) & 1) && 2 + b < nr) v ^= C.col[2 + b];
            hi64[size_t(k) * size_t(slots) + size_t(sl)] = v;
            wk[size_t(k) * size_t(slots) + size_t(sl)] = active ? mult : 0.f;
        }
    }
    cudaError_t e;
    const size_t n_rec = size_t(S) * size_t(slots);
    const size_t word = wide ? sizeof(uint64_t) : sizeof(uint32_t);
    if ((e = cudaMalloc(&w.slot_cone, scone.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(&w.warp_graph, wgraph.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(&w.rec_hi, n_rec * word)) != cudaSuccess ||
        (e = cudaMalloc(&w.rec_wk, n_rec * sizeof(float))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc");
    if (wide) {
        e = cudaMemcpy(w.rec_hi, hi64.data(), n_rec * word, cudaMemcpyHostToDevice);
    } else {
        // at most 32 cut bits in every cone: the high halves are zero
        std::vector<uint32_t> hi32(n_rec);
        for (size_t r = 0; r < n_rec; ++r) hi32[r] = uint32_t(hi64[r]);
        e = cudaMemcpy(w.rec_hi, hi32.data(), n_rec * word, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(w.rec_wk, wk.data(), n_rec * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(w.slot_cone, scone.data(), scone.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(w.warp_graph, wgraph.data(), wgraph.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    return QAOA_OK;
}

// The depth-1 kernel's list (every cone with inner part {u, v}, mixed by the
// only layer): per graph, the shell blocks of its cones back to back, each
// as (c_0 | c_1 << 8 | c_2 << 16 | c_3 << 24, W) with c_a the cut value of
// amplitude a = z_u + 2 z_v of the block (up to the relabelling below) and
// W = +-multiplicity x orbit size x 2^-n rounded once to float; slot s of a
// graph takes its blocks 16 s .. 16 s + 15, and every graph starts on a
// fresh warp (padding: zero weight).
int build_p1_work(const std::vector<DevCone> &hc, const std::vector<uint64_t> &shell_tab,
                  const std::vector<int32_t> &idx, DevWork &w) {
    std::vector<int32_t> order(idx);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return hc[a].graph < hc[b].graph; });
    std::vector<uint2> blocks;  // flat, graph by graph, each graph padded to 32 slots
    std::vector<int32_t> wgraph;
    const size_t per_warp = size_t(kP1Blocks) * 32;
    for (size_t i = 0; i < order.size();) {
        const int32_t g = hc[size_t(order[i])].graph;
        const size_t first = blocks.size();
        for (; i < order.size() && hc[size_t(order[i])].graph == g; ++i) {
            const DevCone &C = hc[size_t(order[i])];
            const uint64_t lo[4] = {0, C.col[0], C.col[1], C.col[0] ^ C.col[1]};
            const double scale = C.weight * std::ldexp(1.0, -C.n);
            for (int64_t beta = 0; beta < C.n_blocks; ++beta) {
                float mult = 0.f;
                const uint64_t word = host_shell_block(C, shell_tab, uint32_t(beta), mult);
                int c[4];
                for (int a = 0; a < 4; ++a) c[a] = __builtin_popcountll(lo[a] ^ word);
                // amplitude order: relabel by f in {X_u, X_v, X_u X_v} (index a -> a
                // xor f) so that the first cut value, against which the kernel
                // shifts C in d/dgamma, is the one nearest the middle of the four;
                // a single flip turns Z_u Z_v into -Z_u Z_v, so W changes sign
                int f = 0, spread = 1 << 30;
                for (int r = 0; r < 4; ++r) {
                    int dev = 0;
                    for (int a = 0; a < 4; ++a) dev = std::max(dev, std::abs(c[a] - c[r]));
                    if (dev < spread) {
                        spread = dev;
                        f = r;
                    }
                }
                uint32_t cnt = 0;
                for (int a = 0; a < 4; ++a) cnt |= uint32_t(c[a ^ f]) << (8 * a);
                const float wf = float(double(mult) * scale) * ((f == 1 || f == 2) ? -1.f : 1.f);
                uint32_t bits;
                std::memcpy(&bits, &wf, sizeof bits);
                blocks.push_back(make_uint2(cnt, bits));
            }
        }
        const size_t n = blocks.size() - first;
        const size_t padded = (n + per_warp - 1) / per_warp * per_warp;
        blocks.resize(first + padded, make_uint2(0u, 0u));
        wgraph.insert(wgraph.end(), padded / per_warp, g);
    }
    const int64_t slots = int64_t(blocks.size() / kP1Blocks);
    w.slots = slots;
    w.warps = slots / 32;
    w.n = int32_t(order.size());
    if (slots == 0) return QAOA_OK;
    // records [k][slot]: block k of slot s is flat block 16 s + k
    std::vector<uint2> rec(blocks.size());
    for (int64_t sl = 0; sl < slots; ++sl)
        for (int k = 0; k < kP1Blocks; ++k)
            rec[size_t(k) * size_t(slots) + size_t(sl)] = blocks[size_t(sl) * kP1Blocks + size_t(k)];
    cudaError_t e;
    if ((e = cudaMalloc(&w.warp_graph, wgraph.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(&w.rec_cw, rec.size() * sizeof(uint2))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc");
    e = cudaMemcpy(w.rec_cw, rec.data(), rec.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(w.warp_graph, wgraph.data(), wgraph.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    return QAOA_OK;
}

RegWork as_reg(const qaoa_device_plan *d, const DevWork &w) { return reg_work(d, w); }

int check_device(const qaoa_plan *plan) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != plan->dev->device) {
        set_error("plan was uploaded to device " + std::to_string(plan->dev->device) + ", current device is " +
                  std::to_string(dev));
        return QAOA_E_INVALID;
    }
    return QAOA_OK;
}

int ensure_uploaded(const qaoa_plan *plan) {
    if (!plan->dev) return qaoa_plan_upload(const_cast<qaoa_plan *>(plan));
    return check_device(plan);
}

// Register qubits per thread of the adjoint kernel: the tuned value, else by
// the amount of work.  Five register qubits halve the lane exchanges but need
// 255 registers (2 blocks of 128 threads per SM), so they win on plans that
// keep the SMs busy for several waves (measured at p = 2: 10% faster on four
// random cubic graphs of 2000 vertices, 9% on two random 4-regular ones) and
// lose on small ones (11-28% slower on the 8x8 and 100x100 tori, one to three
// cones).  The untuned choice takes 5 when the 5-qubit work list, at up to 32
// points per warp task, gives at least four waves of 8 warps per SM.
int reg_bits_for(const qaoa_device_plan *d, int64_t n_points) {
    if (d->reg_bits_grad == 4 || d->reg_bits_grad == 5) return d->reg_bits_grad;
    const int64_t tasks = d->reg_g[1].warps * ((n_points + 31) / 32);
    return tasks >= int64_t(sm_count()) * 8 * 4 ? 5 : 4;
}

// Persistent grid: the occupancy-sized grid, or blocks_per_sm per SM if tuned
// (never above the occupancy limit).
int64_t tuned_grid(const qaoa_device_plan *d, int occupancy_grid) {
    if (d->blocks_per_sm <= 0) return occupancy_grid;
    return std::min<int64_t>(occupancy_grid, int64_t(sm_count()) * d->blocks_per_sm);
}

// Large-state cones: per shape, waves of blocks that fit the scratch budget,
// each wave streamed through the shape's pass list.
cudaError_t run_big(const qaoa_device_plan *d, const qaoa_plan *plan, int64_t P, const double *params,
                    const float2 *lut, const float2 *mix, const float *kpow, double *energy, double *grad,
                    double *terms, bool norm, cudaStream_t s) {
    qaoa_device_plan *dm = const_cast<qaoa_device_plan *>(d);
    const int p = plan->p;
    float4 *cs = nullptr;
    float2 *fa = nullptr;  // the adjoint's first-layer coefficient in hi + lo
    cudaError_t e = cudaMallocAsync(&cs, size_t(plan->n_graphs) * P * p * sizeof(float4), s);
    if (e != cudaSuccess) return e;
    if (grad && (e = cudaMallocAsync(&fa, size_t(plan->n_graphs) * P * sizeof(float2), s)) != cudaSuccess) {
        cudaFreeAsync(cs, s);
        return e;
    }
    e = launch_big_prep(params, int64_t(plan->n_graphs) * P, p, cs, fa, s);
    dm->all_launches += 1;
    const bool g = grad != nullptr;
    const int grid = big_grid(g);
    for (const BigShape &bs : d->big) {
        if (e != cudaSuccess) break;
        const bool split = g ? bs.split_g : bs.split_e;
        // the general adjoint keeps psi and lambda; everything else one block per item
        const int64_t block_bytes = (int64_t(1) << bs.n_in) * int64_t(sizeof(float2)) * (g && !split ? 2 : 1);
        const int64_t items = bs.ystart.back() * P;
        const int64_t wave = std::max<int64_t>(1, std::min<int64_t>(items, int64_t(d->big_budget) / block_bytes));
        float2 *scratch = nullptr;
        e = cudaMallocAsync(&scratch, size_t(wave) * block_bytes, s);
        if (e != cudaSuccess) break;
        BigLaunch B{};
        B.cones = d->cones;
        B.cone_ids = bs.d_cones;
        B.ystart = bs.d_ystart;
        B.n_shape = int32_t(bs.cones.size());
        B.n_in = bs.n_in;
        B.P = P;
        B.p = p;
        B.cmax1 = d->cmax1;
        B.lut = lut;
        B.cs = cs;
        B.fa = fa;
        B.mix = mix;
        B.kpow = kpow;
        B.psi = scratch;
        B.lam = g && !split ? scratch + size_t(wave) * (size_t(1) << bs.n_in) : nullptr;
        B.shell = d->shell;
        B.energy = energy;
        B.grad = grad;
        B.terms = terms;
        B.status = d->status;
        B.norm = norm ? 1 : 0;
        const std::vector<BigPass> &passes = g ? bs.grad : bs.fwd;
        for (int64_t i0 = 0; i0 < items && e == cudaSuccess; i0 += wave) {
            B.item0 = i0;
            B.n_items = std::min(wave, items - i0);
            if (split) {
                e = launch_split_wave(B, g, d->chunk_window, dm->all_launches, s);
                continue;
            }
            for (const BigPass &ps : passes) {
                B.pass = ps;
                e = launch_big_pass(B, g, grid, s);
                dm->all_launches += 1;
                if (e != cudaSuccess) break;
            }
        }
        cudaFreeAsync(scratch, s);
    }
    cudaFreeAsync(cs, s);
    if (fa) cudaFreeAsync(fa, s);
    return e;
}

// norm: the observable is the identity instead of Z_u Z_v (energy path only;
// terms then receive sum |psi|^2 per representative and energy is scratch)
int run(const qaoa_plan *plan, int64_t n_points, const double *params, double *energy, double *grad,
        double *terms, cudaStream_t s, bool norm = false) {
    if (!plan || n_points < 1 || !params || !energy) {
        set_error("need a plan, n_points >= 1, params and energy");
        return QAOA_E_INVALID;
    }
    int rc = ensure_uploaded(plan);
    if (rc != QAOA_OK) return rc;
    const qaoa_device_plan *d = plan->dev;
    const int32_t G = plan->n_graphs, p = plan->p;
    float2 *lut = nullptr, *mix = nullptr;
    float *kpow = nullptr;
    if (take_fault(QAOA_FAULT_DEVICE_ALLOC)) {
        set_error("cudaMallocAsync: out of memory (injected by qaoa_inject_fault)");
        return QAOA_E_OOM;
    }
    const size_t nlut = size_t(G) * n_points * p * d->cmax1;
    const size_t nmix = size_t(G) * n_points * p;
    cudaError_t e;
    if ((e = cudaMallocAsync(&lut, nlut * sizeof(float2), s)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    if ((e = cudaMallocAsync(&mix, nmix * sizeof(float2), s)) != cudaSuccess) {
        cudaFreeAsync(lut, s);
        return cuda_fail(e, "cudaMallocAsync");
    }
    if ((e = cudaMallocAsync(&kpow, nmix * kKpow * sizeof(float), s)) != cudaSuccess) {
        cudaFreeAsync(mix, s);
        cudaFreeAsync(lut, s);
        return cuda_fail(e, "cudaMallocAsync");
    }
    const bool wide = d->cmax1 - 1 > 32;
    PrepArgs pa;
    pa.params = params;
    pa.G = G;
    pa.p = p;
    pa.cmax1 = d->cmax1;
    pa.P = n_points;
    pa.half_edges = d->half_edges;
    pa.lut = lut;
    pa.mix = mix;
    pa.kpow = kpow;
    pa.energy = energy;
    pa.grad = grad;
    pa.terms = terms;
    pa.n_reps = d->n_cones;
    e = launch_prep(pa, s);
    qaoa_device_plan *dm = const_cast<qaoa_device_plan *>(d);
    dm->all_launches += 1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (d->timing && e == cudaSuccess) {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaEventRecord(ev0, s);
    }
    // depth 1 (no per-cone terms asked for): the depth-1 kernel over flat block lists
    const bool use_p1 = p == 1 && d->reg_p1.warps > 0 && terms == nullptr && !norm;
    if (e == cudaSuccess && use_p1) {
        RegLaunch L;
        L.n_points = n_points;
        L.p = 1;
        L.cmax1 = d->cmax1;
        L.lut = lut;
        L.mix = mix;
        L.kpow = kpow;
        L.energy = energy;
        L.grad = grad;
        L.terms = nullptr;
        L.status = d->status;
        L.work = as_reg(d, d->reg_p1);
        // points per warp task: as many phase tables as leave room for the
        // resident blocks the kernel is sized for (a tuned value is held to
        // the kernel's shared-memory limit), halved while the tasks would not
        // give every SM 16 warps
        {
            const bool g = grad != nullptr;
            const int64_t row = int64_t(d->cmax1 + 1) * int64_t(sizeof(float2));
            const int64_t fixed = int64_t(reg_p1_smem_bytes(0, d->cmax1, g)) / (kRegBlock / 32);
            const int blocks = g ? kP1GradMinBlocks : kP1EnergyMinBlocks;
            const int64_t fit = (int64_t(smem_per_block(blocks)) / (kRegBlock / 32) - fixed) / row;
            const int64_t cap = (int64_t(kRegMaxSmem) / (kRegBlock / 32) - fixed) / row;
            int64_t jpt = d->points_per_task;
            if (jpt <= 0) {
                jpt = std::min<int64_t>(32, std::max<int64_t>(1, fit));
                while (jpt > 1 && L.work.warps * ((n_points + jpt - 1) / jpt) < int64_t(sm_count()) * 16)
                    jpt = (jpt + 1) / 2;
            }
            jpt = std::max<int64_t>(1, std::min<int64_t>(jpt, cap));
            L.jpt = int32_t(std::min<int64_t>(jpt, n_points));
        }
        const size_t smem = reg_p1_smem_bytes(L.jpt, d->cmax1, grad != nullptr);
        const int64_t tasks = L.work.warps * ((n_points + L.jpt - 1) / L.jpt);
        int64_t grid = std::min<int64_t>(tuned_grid(d, reg_p1_grid(grad != nullptr, smem)), (tasks + 3) / 4);
        e = launch_reg_p1(L, grad != nullptr, int(std::max<int64_t>(grid, 1)), s);
        dm->all_launches += 1;
        if (e == cudaSuccess && !d->big.empty()) e = run_big(d, plan, n_points, params, lut, mix, kpow, energy, grad, terms, norm, s);
    } else if (e == cudaSuccess) {
        RegLaunch L;
        L.n_points = n_points;
        L.p = p;
        // points per warp task: up to 32, phase tables of at most 8 KB per warp,
        // halved while the tasks would not give every SM 16 warps (small
        // plans: more tasks of fewer points); a tuned value is held to the
        // 48 KB of shared memory of 4 warps
        {
            // one point's phase tables, mixer data and kappa powers
            const int64_t row_bytes = int64_t(p) * ((d->cmax1 + 1) * int64_t(sizeof(float2)) + kRegKpow * int64_t(sizeof(float)));
            const int rgi = reg_bits_for(d, n_points) - 4;
            const int64_t warps = grad ? d->reg_g[rgi].warps : d->reg_e.warps;
            int64_t jpt = d->points_per_task;
            if (jpt <= 0) {
                jpt = std::min<int64_t>(32, std::max<int64_t>(1, 8192 / row_bytes));
                while (jpt > 1 && warps * ((n_points + jpt - 1) / jpt) < int64_t(sm_count()) * 16) jpt = (jpt + 1) / 2;
            }
            jpt = std::min<int64_t>(jpt, std::max<int64_t>(1, 12288 / row_bytes));
            L.jpt = int32_t(std::min<int64_t>(jpt, n_points));
        }
        const size_t smem = reg_smem_bytes(L.jpt, p, d->cmax1, grad != nullptr);
        const int64_t tasks_per = (n_points + L.jpt - 1) / L.jpt;
        L.cmax1 = d->cmax1;
        L.lut = lut;
        L.mix = mix;
        L.kpow = kpow;
        L.energy = energy;
        L.grad = grad;
        L.terms = terms;
        L.status = d->status;
        L.norm = norm && !grad ? 1 : 0;
        if (grad) {
            const int rg = reg_bits_for(d, n_points);
            L.work = as_reg(d, d->reg_g[rg - 4]);
            if (L.work.warps > 0) {
                int64_t grid = std::min<int64_t>(tuned_grid(d, reg_grad_grid(wide, smem, p, rg)),
                                                 (L.work.warps * tasks_per + 3) / 4);
                e = launch_reg_grad(L, wide, rg, int(std::max<int64_t>(grid, 1)), s);
            }
        } else {
            L.work = as_reg(d, d->reg_e);
            if (L.work.warps > 0) {
                int64_t grid = std::min<int64_t>(tuned_grid(d, reg_energy_grid(wide, smem)), (L.work.warps * tasks_per + 3) / 4);
                e = launch_reg_energy(L, wide, int(std::max<int64_t>(grid, 1)), s);
            }
        }
        if (L.work.warps > 0) dm->all_launches += 1;
        if (e == cudaSuccess && !d->big.empty()) e = run_big(d, plan, n_points, params, lut, mix, kpow, energy, grad, terms, norm, s);
    }
    if (ev0) {
        cudaEventRecord(ev1, s);
        dm->events.emplace_back(ev0, ev1);
    }
    cudaFreeAsync(kpow, s);
    cudaFreeAsync(mix, s);
    cudaFreeAsync(lut, s);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return QAOA_OK;
}

}  // namespace

extern "C" void qaoa_device_release(qaoa_plan *plan) {
    if (!plan || !plan->dev) return;
    qaoa_device_plan *d = plan->dev;
    int cur = -1;
    cudaGetDevice(&cur);
    if (d->device >= 0) cudaSetDevice(d->device);
    cudaFree(d->cones);
    free_work(d->reg_e);
    free_work(d->reg_g[0]);
    free_work(d->reg_g[1]);
    free_work(d->reg_p1);
    for (auto &bs : d->big) {
        cudaFree(bs.d_cones);
        cudaFree(bs.d_ystart);
    }
    cudaFree(d->half_edges);
    cudaFree(d->status);
    cudaFree(d->shell);
    for (auto &pr : d->events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (cur >= 0) cudaSetDevice(cur);
    delete d;
    plan->dev = nullptr;
}

extern "C" int qaoa_plan_upload(qaoa_plan *plan) {
    if (!plan) {
        set_error("plan is NULL");
        return QAOA_E_INVALID;
    }
    if (plan->dev) return check_device(plan);
    std::vector<DevCone> hc(plan->cones.size());
    std::vector<uint64_t> shell_tab;
    int32_t cmax = 0;
    std::vector<int32_t> reg_idx;
    int64_t n_big = 0;
    for (size_t i = 0; i < plan->cones.size(); ++i) {
        const Cone &c = plan->cones[i];
        DevCone &d = hc[i];
        std::memset(&d, 0, sizeof d);
        d.graph = c.graph;
        d.n = c.n;
        d.n_in = c.n_in;
        for (int l = 0; l < QAOA_MAX_P; ++l) d.k[l] = c.k[l];
        d.weight = double(c.weight);
        d.rep = int64_t(i);
        // cut word bits: an edge of weight w owns |w| bits; the bits of negative
        // edges are XORed in as a constant (neg), since -b = (b xor 1) - 1 for a
        // cut bit b and the constant only adds a global phase
        int32_t bit = 0;
        for (size_t e = 0; e < c.ea.size(); ++e) {
            const int32_t w = c.ew[e], aw = w < 0 ? -w : w;
            const uint64_t mask = (aw >= 64 ? ~0ull : ((1ull << aw) - 1)) << bit;
            d.col[c.ea[e]] |= mask;
            d.col[c.eb[e]] |= mask;
            if (w < 0) d.neg |= mask;
            bit += aw;
        }
        d.m = bit;
        for (int l = 0; l < QAOA_MAX_P; ++l)
            for (int q = 0; q < c.k[l]; ++q) d.pw[l] ^= d.col[q];
        d.n_blocks = c.n_blocks;
        d.n_cls = int32_t(c.shell_classes.size());
        d.cls_off = int32_t(shell_tab.size());
        if (!c.blk_counts.empty()) {
            // explicit block list (merged blocks): (shell word, multiplicity bits) per block
            d.n_cls = -1;
            for (size_t b = 0; b < c.blk_counts.size(); ++b) {
                uint64_t word = d.neg;
                for (size_t k = 0; k < c.shell_classes.size(); ++k)
                    for (int t = 0; t < c.blk_counts[b][k]; ++t) word ^= d.col[c.shell_classes[k][size_t(t)]];
                const float f = float(c.blk_weight[b]);
                uint32_t bits;
                std::memcpy(&bits, &f, sizeof bits);
                shell_tab.push_back(word);
                shell_tab.push_back(bits);
            }
        } else if (d.neg) {
            // the negative edges' constant enters every cut word once, through a
            // class of no qubits in front of the shell classes (one block, weight 1)
            const float one = 1.f;
            uint32_t one_bits;
            std::memcpy(&one_bits, &one, sizeof one_bits);
            shell_tab.push_back(0);
            shell_tab.push_back(d.neg);
            shell_tab.push_back(one_bits);
            d.n_cls += 1;
        }
        for (const auto &cls : c.blk_counts.empty() ? c.shell_classes : std::vector<std::vector<int32_t>>()) {
            const size_t sz = cls.size();
            shell_tab.push_back(sz);
            uint64_t pm = 0;
            shell_tab.push_back(0);
            for (size_t a = 0; a < sz; ++a) {
                pm ^= d.col[cls[a]];
                shell_tab.push_back(pm);
            }
            double bin = 1.0;  // binomial(sz, nc), exact in double for sz <= 32
            for (size_t nc = 0; nc <= sz; ++nc) {
                const float f = float(bin);
                uint32_t bits;
                std::memcpy(&bits, &f, sizeof bits);
                shell_tab.push_back(bits);
                bin = bin * double(sz - nc) / double(nc + 1);
            }
        }
        cmax = std::max(cmax, d.m);
        if (c.n_in <= kRegMaxInner)
            reg_idx.push_back(int32_t(i));
        else
            ++n_big;
    }
    auto *d = new qaoa_device_plan;
    for (size_t i = 0; i < plan->cones.size(); ++i) {
        const Cone &c = plan->cones[i];
        if (c.n_in <= kRegMaxInner) continue;
        std::vector<int32_t> kv(c.k, c.k + plan->p);
        BigShape *shape = nullptr;
        for (auto &bs : d->big)
            if (bs.n_in == c.n_in && bs.k == kv) shape = &bs;
        if (!shape) {
            d->big.emplace_back();
            shape = &d->big.back();
            shape->n_in = c.n_in;
            shape->k = kv;
            shape->ystart.push_back(0);
            const bool general = (plan->flags & QAOA_BIG_GENERAL) != 0;
            shape->split_e = !general && split_ok(c.n_in, plan->p, kv.data(), false);
            shape->split_g = !general && split_ok(c.n_in, plan->p, kv.data(), true);
            shape->fwd = big_forward_passes(c.n_in, plan->p, kv.data());
            shape->grad = big_grad_passes(c.n_in, plan->p, kv.data());
        }
        shape->cones.push_back(int32_t(i));
        shape->ystart.push_back(shape->ystart.back() + c.n_blocks);
    }
    cudaGetDevice(&d->device);
    d->n_cones = int64_t(hc.size());
    d->cmax1 = cmax + 1;
    d->n_big = n_big;
    plan->dev = d;
    cudaError_t e;
    int rc = QAOA_OK;
    if (!hc.empty()) {
        if ((e = cudaMalloc(&d->cones, hc.size() * sizeof(DevCone))) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMalloc");
        } else if ((e = cudaMemcpy(d->cones, hc.data(), hc.size() * sizeof(DevCone), cudaMemcpyHostToDevice)) !=
                   cudaSuccess) {
            rc = cuda_fail(e, "cudaMemcpy");
        }
    }
    for (auto &bs : d->big) {
        if (rc != QAOA_OK) break;
        if ((e = cudaMalloc(&bs.d_cones, bs.cones.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc(&bs.d_ystart, bs.ystart.size() * sizeof(int64_t))) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMalloc");
        } else {
            cudaMemcpy(bs.d_cones, bs.cones.data(), bs.cones.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
            cudaMemcpy(bs.d_ystart, bs.ystart.data(), bs.ystart.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        }
    }
    if (rc == QAOA_OK) {
        if (shell_tab.empty()) shell_tab.push_back(0);
        if ((e = cudaMalloc(&d->shell, shell_tab.size() * sizeof(uint64_t))) != cudaSuccess)
            rc = cuda_fail(e, "cudaMalloc");
        else
            cudaMemcpy(d->shell, shell_tab.data(), shell_tab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    }
    const bool wide = cmax > 32;  // the kernels' cut-word width (as at launch)
    if (rc == QAOA_OK) rc = build_work(hc, shell_tab, reg_idx, kRegBitsEnergy, wide, d->reg_e);
    if (rc == QAOA_OK) rc = build_work(hc, shell_tab, reg_idx, 4, wide, d->reg_g[0]);
    if (rc == QAOA_OK) rc = build_work(hc, shell_tab, reg_idx, 5, wide, d->reg_g[1]);
    // depth 1 with every register cone mixing qubits 0 and 1 only (its inner
    // part): the depth-1 kernel's list
    bool p1 = plan->p == 1 && !reg_idx.empty();
    for (int32_t i : reg_idx) p1 = p1 && hc[size_t(i)].n_in == 2 && hc[size_t(i)].k[0] == 2;
    if (rc == QAOA_OK && p1) rc = build_p1_work(hc, shell_tab, reg_idx, d->reg_p1);
    if (rc == QAOA_OK) {
        std::vector<double> half(size_t(plan->n_graphs));
        for (int32_t g = 0; g < plan->n_graphs; ++g) half[g] = 0.5 * double(plan->weight_sum[g]);
        if ((e = cudaMalloc(&d->half_edges, half.size() * sizeof(double))) != cudaSuccess)
            rc = cuda_fail(e, "cudaMalloc");
        else
            cudaMemcpy(d->half_edges, half.data(), half.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (rc == QAOA_OK) {
        if ((e = cudaMalloc(&d->status, sizeof(int32_t))) != cudaSuccess)
            rc = cuda_fail(e, "cudaMalloc");
        else if ((e = cudaMemset(d->status, 0, sizeof(int32_t))) != cudaSuccess)
            rc = cuda_fail(e, "cudaMemset");
    }
    if (rc == QAOA_OK && !d->big.empty() && (e = split_prepare()) != cudaSuccess) rc = cuda_fail(e, "kernel attributes");
    if (rc == QAOA_OK && (e = reg_prepare()) != cudaSuccess) rc = cuda_fail(e, "kernel attributes");
    // commit qaoa_energy_noalloc's static scratch on this device now, during set-up
    // (not fatal here: that entry point repeats the lookup and reports a failure)
    if (rc == QAOA_OK) {
        const std::string keep = qaoa_last_error();
        if (noalloc_prepare() != QAOA_OK) set_error(keep);
    }
    if (rc == QAOA_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) rc = cuda_fail(e, "upload");
    if (rc != QAOA_OK) qaoa_device_release(plan);
    return rc;
}

extern "C" int qaoa_plan_info(const qaoa_plan *plan, qaoa_plan_info_t *info) {
    if (!plan || !info) {
        set_error("plan or info is NULL");
        return QAOA_E_INVALID;
    }
    std::memset(info, 0, sizeof *info);
    info->p = plan->p;
    info->n_graphs = plan->n_graphs;
    for (int64_t m : plan->n_edges) info->n_edges_total += m;
    info->n_reps = int64_t(plan->cones.size());
    info->orbits_complete = 1;
    for (const auto &o : plan->orbits) info->orbits_complete &= o.complete ? 1 : 0;
    int64_t n_reg = 0, n_reg_p1 = 0;
    for (const Cone &c : plan->cones) {
        if (c.n_in <= kRegMaxInner) {
            ++n_reg;
            if (c.n_in == 2 && c.k[0] == 2) ++n_reg_p1;
        }
        info->max_qubits = std::max(info->max_qubits, c.n);
        info->max_inner = std::max(info->max_inner, c.n_in);
        info->max_edges = std::max(info->max_edges, int32_t(c.ea.size()));
        info->amps_per_point += std::ldexp(1.0, c.n);
        if (c.n_in > kRegMaxInner) {
            info->n_big++;
            const bool general = (plan->flags & QAOA_BIG_GENERAL) != 0;
            if (general || !split_ok(c.n_in, plan->p, c.k, false)) info->n_big_general_energy++;
            if (general || !split_ok(c.n_in, plan->p, c.k, true)) info->n_big_general_grad++;
        }
    }
    info->depth1_kernel = plan->p == 1 && n_reg > 0 && n_reg_p1 == n_reg ? 1 : 0;
    info->on_device = plan->dev ? 1 : 0;
    info->t_orbits_s = plan->t_orbits;
    info->t_cones_s = plan->t_cones;
    return QAOA_OK;
}

extern "C" int qaoa_energy(const qaoa_plan *plan, int64_t n_points, const double *params_dev, double *energy_dev,
                           double *terms_dev, qaoa_stream_t stream) {
    return run(plan, n_points, params_dev, energy_dev, nullptr, terms_dev, (cudaStream_t)stream);
}

extern "C" int qaoa_norms(const qaoa_plan *plan, int64_t n_points, const double *params_dev, double *norms_dev,
                          qaoa_stream_t stream) {
    if (!plan || n_points < 1 || !params_dev || !norms_dev) {
        set_error("need a plan, n_points >= 1, params and norms");
        return QAOA_E_INVALID;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    double *scratch = nullptr;  // the energy output of the identity observable, unused
    cudaError_t e = cudaMallocAsync(&scratch, size_t(plan->n_graphs) * size_t(n_points) * sizeof(double), s);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? QAOA_E_OOM : QAOA_E_CUDA;
    }
    const int rc = run(plan, n_points, params_dev, scratch, nullptr, norms_dev, s, true);
    cudaFreeAsync(scratch, s);
    return rc;
}

extern "C" int qaoa_energy_grad(const qaoa_plan *plan, int64_t n_points, const double *params_dev,
                                double *energy_dev, double *grad_dev, double *terms_dev, qaoa_stream_t stream) {
    if (!grad_dev) {
        set_error("grad_dev is NULL");
        return QAOA_E_INVALID;
    }
    return run(plan, n_points, params_dev, energy_dev, grad_dev, terms_dev, (cudaStream_t)stream);
}

extern "C" int qaoa_cut_table(const qaoa_plan *plan, int64_t rep, uint8_t *out_dev, qaoa_stream_t stream) {
    if (!plan || rep < 0 || rep >= int64_t(plan->cones.size()) || !out_dev) {
        set_error("bad plan, representative index or output pointer");
        return QAOA_E_INVALID;
    }
    int rc = ensure_uploaded(plan);
    if (rc != QAOA_OK) return rc;
    cudaError_t e =
        launch_cut_table(plan->dev->cones + rep, out_dev, plan->cones[rep].n, plan->dev->status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cut table launch");
    return QAOA_OK;
}

extern "C" int qaoa_device_status(const qaoa_plan *plan, int32_t *status) {
    if (!plan || !status) {
        set_error("plan or status is NULL");
        return QAOA_E_INVALID;
    }
    if (!plan->dev) {
        *status = 0;
        return QAOA_OK;
    }
    int rc = check_device(plan);
    if (rc != QAOA_OK) return rc;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    int32_t v = 0;
    if ((e = cudaMemcpy(&v, plan->dev->status, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    cudaMemset(plan->dev->status, 0, sizeof(int32_t));
    *status = v;
    return QAOA_OK;
}

extern "C" int qaoa_plan_timing(qaoa_plan *plan, int32_t enable) {
    if (!plan) {
        set_error("plan is NULL");
        return QAOA_E_INVALID;
    }
    int rc = ensure_uploaded(plan);
    if (rc != QAOA_OK) return rc;
    plan->dev->timing = enable != 0;
    return QAOA_OK;
}

extern "C" int qaoa_kernel_time(qaoa_plan *plan, double *ms, int64_t *launches, int64_t *all_launches) {
    if (!plan) {
        set_error("plan is NULL");
        return QAOA_E_INVALID;
    }
    double total = 0.0;
    int64_t count = 0, all = 0;
    if (plan->dev) {
        qaoa_device_plan *d = plan->dev;
        for (auto &pr : d->events) {
            cudaError_t e = cudaEventSynchronize(pr.second);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
            float t = 0.f;
            cudaEventElapsedTime(&t, pr.first, pr.second);
            total += t;
            ++count;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        d->events.clear();
        all = d->all_launches;
        d->all_launches = 0;
    }
    if (ms) *ms = total;
    if (launches) *launches = count;
    if (all_launches) *all_launches = all;
    return QAOA_OK;
}

extern "C" int qaoa_plan_set_tuning(qaoa_plan *plan, const qaoa_tuning_t *t) {
    if (!plan || !t || t->points_per_task < 0 || t->blocks_per_sm < 0 || t->big_scratch_bytes < 0 ||
        (t->reg_bits_grad != 0 && t->reg_bits_grad != 4 && t->reg_bits_grad != 5) ||
        (t->chunk_window != 0 && (t->chunk_window < 6 || t->chunk_window > 10))) {
        set_error("bad plan or tuning values");
        return QAOA_E_INVALID;
    }
    int rc = ensure_uploaded(plan);
    if (rc != QAOA_OK) return rc;
    plan->dev->points_per_task = t->points_per_task;
    plan->dev->blocks_per_sm = t->blocks_per_sm;
    plan->dev->big_budget = t->big_scratch_bytes > 0 ? size_t(t->big_scratch_bytes) : size_t(1) << 30;
    plan->dev->reg_bits_grad = t->reg_bits_grad;
    plan->dev->chunk_window = t->chunk_window > 0 ? t->chunk_window : 10;
    return QAOA_OK;
}

extern "C" int qaoa_plan_get_tuning(const qaoa_plan *plan, qaoa_tuning_t *t) {
    if (!plan || !t) {
        set_error("plan or tuning is NULL");
        return QAOA_E_INVALID;
    }
    t->points_per_task = plan->dev ? plan->dev->points_per_task : 0;
    t->blocks_per_sm = plan->dev ? plan->dev->blocks_per_sm : 0;
    t->big_scratch_bytes = plan->dev ? int64_t(plan->dev->big_budget) : int64_t(1) << 30;
    t->reg_bits_grad = plan->dev ? plan->dev->reg_bits_grad : 0;
    t->chunk_window = plan->dev ? plan->dev->chunk_window : 10;
    return QAOA_OK;
}

struct qaoa_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int qaoa_graph_create(qaoa_plan *plan, int64_t n_points, const double *params_dev, double *energy_dev,
                                 double *grad_dev, double *terms_dev, qaoa_graph **out) {
    if (!out) {
        set_error("out is NULL");
        return QAOA_E_INVALID;
    }
    *out = nullptr;
    if (!plan || n_points < 1 || !params_dev || !energy_dev) {
        set_error("need a plan, n_points >= 1, params and energy");
        return QAOA_E_INVALID;
    }
    int rc = ensure_uploaded(plan);
    if (rc != QAOA_OK) return rc;
    const bool timing = plan->dev->timing;
    plan->dev->timing = false;  // no event records inside the graph
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        plan->dev->timing = timing;
        return cuda_fail(e, "cudaStreamCreate");
    }
    auto *g = new qaoa_graph;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = run(plan, n_points, params_dev, energy_dev, grad_dev, terms_dev, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g->graph);
        if (rc == QAOA_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        rc = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (rc == QAOA_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
    }
    cudaStreamDestroy(cap);
    plan->dev->timing = timing;
    if (rc != QAOA_OK) {
        qaoa_graph_free(g);
        return rc;
    }
    *out = g;
    return QAOA_OK;
}

extern "C" int qaoa_graph_launch(qaoa_graph *graph, qaoa_stream_t stream) {
    if (!graph || !graph->exec) {
        set_error("graph is NULL");
        return QAOA_E_INVALID;
    }
    cudaError_t e = cudaGraphLaunch(graph->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return QAOA_OK;
}

extern "C" void qaoa_graph_free(qaoa_graph *graph) {
    if (!graph) return;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
}
