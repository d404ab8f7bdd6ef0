// C ABI of the batched path (olb_batch_*): many independent lattices advanced
// together by one persistent kernel per time step, K steps per CUDA-graph
// replay.  See oreg_batch_kernels.cuh for the device side.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "oreg.h"
#include "oreg_batch_kernels.cuh"
#include "oreg_launch.h"
#include "oreg_lattice.h"

using namespace oreg;

namespace {

olb_status bfail(olb_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error_message(buf);
    return st;
}

olb_status bcuda(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) (void)cudaGetLastError();  // not sticky: clear it
    return bfail(e == cudaErrorMemoryAllocation ? OLB_ERR_NOMEM : OLB_ERR_CUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

#define B_CUDA(call, what)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda(e_, what);      \
    } while (0)

#define BDISPATCH(storage, fn, ...)                                     \
    ((storage) == OLB_F64   ? fn##_f64(__VA_ARGS__)                     \
     : (storage) == OLB_F32 ? fn##_f32(__VA_ARGS__)                     \
     : (storage) == OLB_F16_SHIFTED ? fn##_f16(__VA_ARGS__)             \
                                    : fn##_bf16(__VA_ARGS__))

// Slots (one kernel and one constant class each) a batch tracks before it
// compacts its slot list; work-item groups are (slot, parity class).
constexpr int MAX_SLOTS = 64;
constexpr int NGROUPS = 2 * MAX_SLOTS;
constexpr int SIDE_STREAMS = 8;  // capture streams for the slots of a step

// (walls, equilibrium kind, collision) of a lattice: its batch kernel
int combo_index(const olb_lattice *L) {
    const int walls = L->p.boundary == OLB_BOUNDARY_WALLS_X;
    return (walls * 3 + kernel_eq(&L->p)) * 2 + L->p.coll;
}

struct Member {
    olb_lattice *lat;
    long long g_base, g_end;  // active global steps [g_base, g_end)
    long long t_base;         // lattice time at g_base
    int slot;
};

// A slot: kernel combination and the class constants (lam zeroed).
struct Slot {
    int combo;
    std::vector<char> k;
};

// The collision constants a lattice's batch kernel takes, with lam (per
// lattice, from the descriptor) zeroed: the lattice's constant class.
std::vector<char> class_constants(const olb_lattice *L) {
    std::vector<char> out;
    if (L->p.storage == OLB_F64) {
        CollConst<double> k = L->kd;
        k.lam = 0.0;
        out.assign(reinterpret_cast<const char *>(&k), reinterpret_cast<const char *>(&k) + sizeof k);
    } else {
        CollConst<float> k = L->kf;
        k.lam = 0.0f;
        out.assign(reinterpret_cast<const char *>(&k), reinterpret_cast<const char *>(&k) + sizeof k);
    }
    return out;
}

template <typename C>
void fill_desc(void *dst, const Member &m, C lam) {
    BatchDesc<C> d;
    std::memset(&d, 0, sizeof d);
    const olb_lattice *L = m.lat;
    d.mem = L->mem;
    d.nx = L->p.nx;
    d.ny = L->p.ny;
    d.pitch = L->pitch;
    d.eq = L->p.eq;
    d.coll = L->p.coll;
    d.plane = L->plane;
    d.buf_elems = L->buf_elems;
    d.t_base = m.t_base;
    d.g_base = m.g_base;
    d.g_end = m.g_end;
    d.sr = L->sr;
    d.lam = lam;
    std::memcpy(dst, &d, sizeof d);
}

}  // namespace

struct olb_batch {
    olb_batch_params p;
    cudaStream_t stream;
    bool own_stream;
    int num_sms;
    int grid, block;
    size_t desc_size;
    // device tables
    char *d_descs;
    int4 *d_items;
    int *d_groups;          // item offsets of the (slot, parity class) groups
    long long *d_g;
    // Pinned staging of the table uploads, two buffers used alternately: an
    // upload copies the host tables into one and enqueues its copies on the
    // batch stream, so joining and leaving never wait for running rounds
    // (the copies land between rounds in stream order); a buffer is refilled
    // only after the copies issued from it two uploads earlier have run.
    char *h_stage[2];
    size_t stage_bytes[2];
    cudaEvent_t stage_done[2];
    bool stage_pending[2];
    int next_stage;
    // host mirrors
    std::vector<Member> members;
    std::vector<Slot> slots;   // slots in launch order (kept while the graph is valid)
    std::vector<char> h_descs;
    std::vector<int4> h_items;
    std::vector<int> h_groups;  // NGROUPS + 1 entries
    long long G;            // global step counter at the start of the next round
    bool captured;
    int graph_slots;        // slots the captured graph launches
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    // Used while capturing only: with several slots, each slot's launches go
    // to one of these streams, forked from and joined back into the batch
    // stream, so that the graph runs the kernels of different slots (disjoint
    // lattices) side by side instead of one after another.
    cudaStream_t side[SIDE_STREAMS];
    cudaEvent_t fork_ev, join_ev[SIDE_STREAMS];
    int nside;              // side streams created so far
    cudaEvent_t wait_ev;    // olb_batch_wait_for (created on first use)
};

namespace {

void drop_graph(olb_batch *b) {
    // replays still queued finish before the executable graph goes away
    if (b->exec) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->captured = false;
}

// Slot of a member: an existing slot with its kernel and constants, else a
// new one at the end (the captured graph then lacks it and is dropped).  When
// the list is full, slots no member uses are removed (renumbering the rest)
// and the graph is dropped too.
int slot_for(olb_batch *b, const olb_lattice *L) {
    const int combo = combo_index(L);
    const std::vector<char> k = class_constants(L);
    for (size_t s = 0; s < b->slots.size(); ++s)
        if (b->slots[s].combo == combo && b->slots[s].k == k) return (int)s;
    if ((int)b->slots.size() == MAX_SLOTS) {
        std::vector<Slot> kept;
        for (Member &m : b->members) {
            int found = -1;
            for (size_t s = 0; s < kept.size(); ++s)
                if (kept[s].combo == b->slots[m.slot].combo && kept[s].k == b->slots[m.slot].k)
                    found = (int)s;
            if (found < 0) {
                kept.push_back(b->slots[m.slot]);
                found = (int)kept.size() - 1;
            }
            m.slot = found;
        }
        b->slots.swap(kept);
        drop_graph(b);
        for (size_t s = 0; s < b->slots.size(); ++s)
            if (b->slots[s].combo == combo && b->slots[s].k == k) return (int)s;
        if ((int)b->slots.size() == MAX_SLOTS) return -1;
    }
    b->slots.push_back(Slot{combo, k});
    if (b->captured && (int)b->slots.size() > b->graph_slots) drop_graph(b);
    return (int)b->slots.size() - 1;
}

olb_status upload(olb_batch *b) {
    const size_t nm = b->members.size();
    b->h_descs.assign(nm * b->desc_size, 0);
    std::vector<std::vector<int4>> per_group(NGROUPS);
    for (size_t j = 0; j < nm; ++j) {
        const Member &m = b->members[j];
        const olb_lattice *L = m.lat;
        if (L->p.storage == OLB_F64) fill_desc<double>(&b->h_descs[j * b->desc_size], m, L->kd.lam);
        else fill_desc<float>(&b->h_descs[j * b->desc_size], m, L->kf.lam);
        const int cls = (int)((m.t_base - m.g_base) & 1);
        const int grp = m.slot * 2 + cls;
        // item: (member, first vector, 0, warp passes of 32 vectors)
        const int passes = (int)warp_passes(L->pitch, L->p.ny, L->V);
        const int R = b->p.item_passes;
        for (int q = 0; q < passes; q += R)
            per_group[grp].push_back(make_int4((int)j, q * 32, 0, std::min(R, passes - q)));
    }
    b->h_items.clear();
    for (int q = 0; q < NGROUPS; ++q) {
        b->h_groups[q] = (int)b->h_items.size();
        b->h_items.insert(b->h_items.end(), per_group[q].begin(), per_group[q].end());
    }
    b->h_groups[NGROUPS] = (int)b->h_items.size();
    if ((long long)b->h_items.size() > b->p.max_items)
        return bfail(OLB_ERR_NOMEM, "batch work items %zu exceed max_items %lld", b->h_items.size(),
                     (long long)b->p.max_items);
    // stage the three tables in one pinned buffer and copy them in stream order
    const size_t nd = b->h_descs.size(), ni = b->h_items.size() * sizeof(int4),
                 ng = (NGROUPS + 1) * sizeof(int);
    const size_t off_i = (nd + 15) / 16 * 16, off_g = off_i + ni, total = off_g + ng;
    const int s = b->next_stage;
    if (b->stage_pending[s])
        B_CUDA(cudaEventSynchronize(b->stage_done[s]), "waiting for an earlier table upload");
    b->stage_pending[s] = false;
    if (b->stage_bytes[s] < total) {
        if (b->h_stage[s]) cudaFreeHost(b->h_stage[s]);
        b->h_stage[s] = nullptr;
        b->stage_bytes[s] = 0;
        const size_t cap = std::max(total, 2 * b->stage_bytes[s ^ 1]);
        B_CUDA(cudaMallocHost(&b->h_stage[s], cap), "allocating pinned table staging");
        b->stage_bytes[s] = cap;
    }
    char *h = b->h_stage[s];
    if (nd) std::memcpy(h, b->h_descs.data(), nd);
    if (ni) std::memcpy(h + off_i, b->h_items.data(), ni);
    std::memcpy(h + off_g, b->h_groups.data(), ng);
    if (nd)
        B_CUDA(cudaMemcpyAsync(b->d_descs, h, nd, cudaMemcpyHostToDevice, b->stream),
               "uploading batch descriptors");
    if (ni)
        B_CUDA(cudaMemcpyAsync(b->d_items, h + off_i, ni, cudaMemcpyHostToDevice, b->stream),
               "uploading batch items");
    B_CUDA(cudaMemcpyAsync(b->d_groups, h + off_g, ng, cudaMemcpyHostToDevice, b->stream),
           "uploading item groups");
    B_CUDA(cudaEventRecord(b->stage_done[s], b->stream), "recording table upload");
    b->stage_pending[s] = true;
    b->next_stage = s ^ 1;
    return OLB_OK;
}

__global__ void k_batch_advance(long long *g, int K) { *g += K; }

// The side streams (and their events) of a capture over nside of them.
olb_status ensure_side(olb_batch *b, int nside) {
    if (!b->fork_ev)
        B_CUDA(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming), "creating capture events");
    while (b->nside < nside) {
        const int i = b->nside;
        B_CUDA(cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking), "creating a capture stream");
        const cudaError_t e = cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaStreamDestroy(b->side[i]);
            b->side[i] = nullptr;
            return bcuda(e, "creating capture events");
        }
        ++b->nside;
    }
    return OLB_OK;
}

// Captures one round: K steps of every slot, then the counter increment.
// With one slot its launches stay on the batch stream; with several, slot s
// goes to side stream s mod S (S = min(slots, SIDE_STREAMS)), forked from the
// batch stream before the first step and joined back before the increment,
// so each slot's steps stay in order while different slots overlap.
olb_status capture(olb_batch *b) {
    std::vector<BatchSlot> slots(b->slots.size());
    for (size_t s = 0; s < b->slots.size(); ++s) slots[s] = BatchSlot{b->slots[s].combo, b->slots[s].k.data()};
    const int nslots = (int)slots.size();
    const int nside = nslots > 1 ? std::min(nslots, SIDE_STREAMS) : 0;
    if (nside) {
        const olb_status st = ensure_side(b, nside);
        if (st != OLB_OK) return st;
    }
    BatchLaunch a{};
    a.descs = b->d_descs;
    a.items = b->d_items;
    a.groups = b->d_groups;
    a.g = b->d_g;
    a.layout = b->p.layout;
    a.grid = b->grid;
    a.block = b->block;
    a.slots = slots.data();
    B_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
           "beginning graph capture");
    cudaError_t e = cudaSuccess;
    int forked = 0;  // side streams that joined the capture
    if (nside) {
        e = cudaEventRecord(b->fork_ev, b->stream);
        while (forked < nside && e == cudaSuccess) {
            e = cudaStreamWaitEvent(b->side[forked], b->fork_ev, 0);
            if (e == cudaSuccess) ++forked;
        }
    }
    for (int k = 0; k < b->p.steps_per_launch && e == cudaSuccess; ++k) {
        a.k = k;
        if (!nside) {
            a.first_slot = 0;
            a.nslots = nslots;
            a.stream = b->stream;
            e = BDISPATCH(b->p.storage, batch_step, a);
        } else {
            for (int s = 0; s < nslots && e == cudaSuccess; ++s) {
                a.first_slot = s;
                a.nslots = 1;
                a.stream = b->side[s % nside];
                e = BDISPATCH(b->p.storage, batch_step, a);
            }
        }
    }
    // join every side stream that joined the capture (also after an error,
    // so that the capture can end)
    for (int i = 0; i < forked; ++i) {
        cudaError_t ej = cudaEventRecord(b->join_ev[i], b->side[i]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->stream, b->join_ev[i], 0);
        if (e == cudaSuccess) e = ej;
    }
    if (e == cudaSuccess) {
        k_batch_advance<<<1, 1, 0, b->stream>>>(b->d_g, b->p.steps_per_launch);
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(e, "capturing batch steps");
    }
    if (e2 != cudaSuccess) return bcuda(e2, "ending graph capture");
    b->graph = g;
    B_CUDA(cudaGraphInstantiate(&b->exec, g, 0), "instantiating batch graph");
    b->captured = true;
    b->graph_slots = nslots;
    return OLB_OK;
}

}  // namespace

extern "C" {

olb_status olb_batch_create(const olb_batch_params *p, olb_batch **out) {
    if (!out) return bfail(OLB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!p) return bfail(OLB_ERR_INVALID, "params is NULL");
    if (p->storage < OLB_F64 || p->storage > OLB_BF16_SHIFTED)
        return bfail(OLB_ERR_INVALID, "unknown storage %d", p->storage);
    if (p->layout != OLB_LAYOUT_AB && p->layout != OLB_LAYOUT_AA)
        return bfail(OLB_ERR_INVALID, "unknown layout %d", p->layout);
    if (p->max_lattices < 1 || p->max_items < 1)
        return bfail(OLB_ERR_INVALID, "max_lattices and max_items must be >= 1");
    if (p->steps_per_launch < 1 || p->steps_per_launch > 10000)
        return bfail(OLB_ERR_INVALID, "steps_per_launch must be in [1, 10000]");
    if (p->warps_per_block < 1 || 32 * p->warps_per_block > BATCH_MAX_THREADS ||
        (p->warps_per_block & (p->warps_per_block - 1)))
        return bfail(OLB_ERR_INVALID, "warps_per_block must be 1, 2 or 4");
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 256)
        return bfail(OLB_ERR_INVALID, "blocks_per_sm must be in [0, 256] (0 = occupancy limit)");
    if (p->item_passes < 0 || p->item_passes > 64)
        return bfail(OLB_ERR_INVALID, "item_passes must be in [0, 64] (0 = %d)",
                     BATCH_ITEM_PASSES);
    olb_batch *b = new (std::nothrow) olb_batch();
    if (!b) return bfail(OLB_ERR_NOMEM, "host allocation of the batch failed");
    b->p = *p;
    if (b->p.item_passes == 0) b->p.item_passes = BATCH_ITEM_PASSES;
    b->desc_size = BDISPATCH(p->storage, batch_desc_size);
    auto bail = [&](olb_status s) {
        olb_batch_destroy(b);
        return s;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bail(bcuda(e, "querying the device"));
    if (p->cuda_stream) {
        b->stream = static_cast<cudaStream_t>(p->cuda_stream);
        b->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(bcuda(e, "creating the stream"));
        b->own_stream = true;
    }
    b->block = 32 * p->warps_per_block;
    int per_sm = p->blocks_per_sm;
    if (per_sm == 0) {
        per_sm = BDISPATCH(p->storage, batch_occupancy, p->layout, b->block);
        if (per_sm < 1) per_sm = 1;
    }
    b->grid = per_sm * b->num_sms;
    e = cudaMalloc(&b->d_descs, (size_t)p->max_lattices * b->desc_size);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, (size_t)p->max_items * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_groups, (NGROUPS + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_g, sizeof(long long));
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
        e = cudaEventCreateWithFlags(&b->stage_done[s], cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(bcuda(e, "allocating batch tables"));
    b->h_groups.assign(NGROUPS + 1, 0);
    e = cudaMemsetAsync(b->d_g, 0, sizeof(long long), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_groups, 0, (NGROUPS + 1) * sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bail(bcuda(e, "clearing batch tables"));
    b->G = 0;
    *out = b;
    return OLB_OK;
}

olb_status olb_batch_add(olb_batch *b, olb_lattice *lat, int64_t nsteps) {
    if (!b || !lat) return bfail(OLB_ERR_INVALID, "batch and lattice must not be NULL");
    if (nsteps < 0) return bfail(OLB_ERR_INVALID, "nsteps must be >= 0");
    if (lat->batch) return bfail(OLB_ERR_STATE, "lattice already belongs to a batch");
    if (lat->t < 0) return bfail(OLB_ERR_STATE, "lattice state not initialised");
    if (lat->f64_coll)
        return bfail(OLB_ERR_INVALID, "OLB_OPT_F64_COLLISION is not available in a batch");
    if (lat->p.storage == OLB_F32 && !lat->comp)
        return bfail(OLB_ERR_INVALID, "batches use the exact conserved sums of FP32 storage: "
                                      "OLB_OPT_COMPENSATED = 0 is not available in a batch");
    if (lat->p.storage != b->p.storage || lat->p.layout != b->p.layout)
        return bfail(OLB_ERR_INVALID, "lattice storage/layout (%d/%d) differ from the batch's (%d/%d)",
                     lat->p.storage, lat->p.layout, b->p.storage, b->p.layout);
    if (lat->stream != b->stream)
        return bfail(OLB_ERR_INVALID, "member lattices must be created on the batch's stream");
    if ((int)b->members.size() >= b->p.max_lattices)
        return bfail(OLB_ERR_NOMEM, "batch holds max_lattices = %d lattices", b->p.max_lattices);
    Member m;
    m.lat = lat;
    m.g_base = b->G;
    m.g_end = b->G + nsteps;
    m.t_base = lat->t;
    // a new slot (kernel or constant class) invalidates the captured graph,
    // which is captured again on the next run
    m.slot = slot_for(b, lat);
    if (m.slot < 0)
        return bfail(OLB_ERR_NOMEM, "batch members use more than %d (kernel, constant class) slots",
                     MAX_SLOTS);
    b->members.push_back(m);
    olb_status st = upload(b);
    if (st != OLB_OK) {
        b->members.pop_back();
        upload(b);
        return st;
    }
    lat->batch = b;
    return OLB_OK;
}

olb_status olb_batch_remove(olb_batch *b, olb_lattice *lat) {
    if (!b || !lat) return bfail(OLB_ERR_INVALID, "batch and lattice must not be NULL");
    auto it = std::find_if(b->members.begin(), b->members.end(),
                           [&](const Member &m) { return m.lat == lat; });
    if (it == b->members.end()) return bfail(OLB_ERR_INVALID, "lattice is not in this batch");
    b->members.erase(it);
    lat->batch = nullptr;
    return upload(b);
}

olb_status olb_batch_run(olb_batch *b, int64_t nrounds) {
    NvtxRange nvtx_("olb_batch_run");
    if (!b) return bfail(OLB_ERR_INVALID, "batch is NULL");
    if (nrounds < 0) return bfail(OLB_ERR_INVALID, "nrounds must be >= 0");
    if (!b->captured) {
        olb_status st = capture(b);
        if (st != OLB_OK) return st;
    }
    const long long K = b->p.steps_per_launch;
    for (int64_t r = 0; r < nrounds; ++r) {
        B_CUDA(cudaGraphLaunch(b->exec, b->stream), "launching batch graph");
        // member times advance by the steps each takes part in this round
        for (Member &m : b->members) {
            const long long lo = std::max(m.g_base, b->G), hi = std::min(m.g_end, b->G + K);
            if (hi > lo) m.lat->t += hi - lo;
        }
        b->G += K;
    }
    return OLB_OK;
}

olb_status olb_batch_wait(olb_batch *b) {
    if (!b) return bfail(OLB_ERR_INVALID, "batch is NULL");
    B_CUDA(cudaStreamSynchronize(b->stream), "waiting for the batch");
    return OLB_OK;
}

olb_status olb_batch_wait_for(olb_batch *b, double seconds) {
    if (!b) return bfail(OLB_ERR_INVALID, "batch is NULL");
    if (!(seconds >= 0) || !(seconds <= 1e6))
        return bfail(OLB_ERR_INVALID, "seconds must be in [0, 1e6] (got %g)", seconds);
    if (!b->wait_ev)
        B_CUDA(cudaEventCreateWithFlags(&b->wait_ev, cudaEventDisableTiming), "creating the wait event");
    B_CUDA(cudaEventRecord(b->wait_ev, b->stream), "recording the wait event");
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(seconds);
    for (;;) {
        const cudaError_t e = cudaEventQuery(b->wait_ev);
        if (e == cudaSuccess) return OLB_OK;
        if (e != cudaErrorNotReady) return bcuda(e, "waiting for the batch");
        if (std::chrono::steady_clock::now() >= until)
            return bfail(OLB_ERR_TIMEOUT, "batch rounds still running after %g s", seconds);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

olb_status olb_batch_remaining(const olb_batch *b, const olb_lattice *lat, int64_t *steps) {
    if (!b || !lat || !steps) return bfail(OLB_ERR_INVALID, "NULL argument");
    for (const Member &m : b->members)
        if (m.lat == lat) {
            *steps = std::max<long long>(0, m.g_end - std::max(m.g_base, b->G));
            return OLB_OK;
        }
    return bfail(OLB_ERR_INVALID, "lattice is not in this batch");
}

int32_t olb_batch_size(const olb_batch *b) { return b ? (int32_t)b->members.size() : 0; }

int64_t olb_batch_work_items(const olb_batch *b) { return b ? (int64_t)b->h_items.size() : 0; }

olb_status olb_batch_destroy(olb_batch *b) {
    if (!b) return OLB_OK;
    olb_status st = OLB_OK;
    if (b->stream) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bcuda(e, "synchronising before destroy");
    }
    for (Member &m : b->members) m.lat->batch = nullptr;
    drop_graph(b);
    if (b->d_descs) cudaFree(b->d_descs);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_groups) cudaFree(b->d_groups);
    if (b->d_g) cudaFree(b->d_g);
    for (int s = 0; s < 2; ++s) {
        if (b->h_stage[s]) cudaFreeHost(b->h_stage[s]);
        if (b->stage_done[s]) cudaEventDestroy(b->stage_done[s]);
    }
    for (int i = 0; i < b->nside; ++i) {
        cudaStreamDestroy(b->side[i]);
        cudaEventDestroy(b->join_ev[i]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->wait_ev) cudaEventDestroy(b->wait_ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return st;
}

}  // extern "C"
