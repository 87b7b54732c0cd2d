// Serving engine: device-resident client generators, an output arena under
// an HBM budget, FIFO admission and continuous batching.  See the contract in
// include/rng.h (rng_server_*).  Clients are split into two lanes (even and
// odd ids), each with its own stream, plan and ticks, so that one lane's
// tick overlaps the other's instead of waiting for its last tiles.
//
// Sample g of a client's sequence is output g / n of stream g % n (n streams
// per client).  A piece of m samples starting at sample c covers columns
// 0 .. m-1 of a row-major window whose column `col` belongs to stream
// (c % n + col) % n: columns below m % n get one output more than the others.
// Each column range maps to at most two contiguous stream ranges (the window
// wraps around stream n-1), so a piece is at most four batch items with
// disjoint stream ranges of one generator, all in the same launch.
//
// One piece per client and tick runs through several of its requests: the
// kernel writes the piece as one virtual window of the client's sequence and
// the piece's output map (runs.h, gen_body.cuh) sends each request's part to
// that request's output in its format.  Every output is placed at a word
// index congruent to its first sample's index modulo 8, so that all of a
// client's outputs agree with any window of its sequence modulo 32 bytes.
#include <algorithm>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "pieces.h"
#include "runs.h"
#include "gbrng.cuh"

namespace gbrng {
namespace {

constexpr uint64_t kGranule = 256;  // arena alignment, bytes
constexpr int kMaxInflight = 2;     // ticks in flight per lane
constexpr int kLanes = 2;           // client c belongs to lane c % kLanes
constexpr int kServeThreads = 512;
constexpr int kServeCtas = 1;  // one CTA per SM: 1664 against 1631 GS/s (two) saturating

// Arena bytes of a request of n samples: its output and room to place it at
// the word phase of its first sample (placement_pad).
inline uint64_t block_bytes(uint64_t n) { return 4 * n + 4 * (kPhaseWords - 1); }


struct Req {
    uint32_t client = 0;
    uint64_t n = 0;      // samples
    int fmt = 0;
    uint64_t start = 0;  // first sample index in the client's sequence
    uint64_t off = 0;    // arena byte offset of the output
    uint64_t block = 0;  // the arena block that holds it (see placement_pad)
    bool admitted = false;
    bool completed = false;
    double done_ms = 0;
};

// An admitted request as the ticks see it (kept beside its client's others,
// so that building a tick reads no hash map).
struct Act {
    uint64_t id;
    uint64_t off;    // arena byte offset
    uint64_t n;      // samples
    uint64_t done;   // samples already scheduled
    uint64_t start;  // first sample index in the client's sequence
    int fmt;
};

// A request waiting for admission (its client and size beside its id, so
// that the admission scan reads no hash map); id kGone once admitted past
// the head.
constexpr uint64_t kGone = ~0ull;
struct Pend {
    uint64_t id;
    uint64_t n;
    uint32_t client;
};

struct Tick {
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> completing;
};

struct Server {
    int kind = 0;
    int device = 0;
    uint32_t n_clients = 0;
    uint64_t streams = 0;
    uint32_t chunk_rows = 0;
    std::vector<rng_handle> gens;
    uint32_t *arena_base = nullptr;
    Arena *arena = nullptr;
    std::vector<uint64_t> cursor;                 // next sample index per client
    std::deque<Pend> pending;  // waiting for admission, in order (admitted
                               // entries past the head are marked kGone)
    size_t n_pending = 0;      // entries not marked
    uint64_t bypassed = 0;        // bytes admitted past the waiting head
    bool rescan = true;           // space released or requests queued since the last scan
    std::vector<char> held;       // admission scan: clients with a request waiting
    std::vector<std::deque<Act>> active;          // admitted, per client, in order
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<Tick> inflight[kLanes];
    std::vector<cudaEvent_t> spare_events;
    std::deque<std::pair<uint64_t, double>> done;  // completed, not yet taken
    std::vector<rng_batch_item> items;
    std::vector<uint64_t> item_map;  // per item: word offset of its piece's format map
    std::vector<uint32_t> maps;      // the tick's format maps
    std::vector<RunReq> run;         // a client's active requests, for run_piece
    rng_plan_handle plan[kLanes] = {};
    cudaStream_t stream[kLanes] = {};
    cudaEvent_t t0 = nullptr;
    uint32_t rr[kLanes] = {};  // round-robin start, per lane
    uint64_t tick_bytes = 0;  // target output per tick (0: chunk_rows alone)
    int plan_threads = kServeThreads, plan_ctas = kServeCtas;  // persistent kernel shape
    uint64_t next_id = 0, n_admitted = 0, n_completed = 0, n_ticks = 0, samples = 0;
};

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~DeviceScope()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

int retire(Server *S)
{
    for (int ln = 0; ln < kLanes; ++ln) {
        while (!S->inflight[ln].empty()) {
            Tick &t = S->inflight[ln].front();
            cudaError_t e = cudaEventQuery(t.ev);
            if (e == cudaErrorNotReady)
                break;
            if (e != cudaSuccess)
                return cuda_status(e);
            float ms = 0;
            cudaEventElapsedTime(&ms, S->t0, t.ev);
            for (uint64_t id : t.completing) {
                Req &q = S->reqs[id];
                q.completed = true;
                q.done_ms = ms;
                S->done.emplace_back(id, (double)ms);
                ++S->n_completed;
            }
            S->spare_events.push_back(t.ev);
            S->inflight[ln].pop_front();
        }
    }
    return RNG_OK;
}

// Requests after a waiting head that admission looks at, per call.
constexpr size_t kLookahead = 1024;

bool admit_one(Server *S, uint64_t id)
{
    Req &q = S->reqs[id];
    uint64_t block = 0;
    if (!S->arena->alloc(block_bytes(q.n), &block))
        return false;
    q.block = block;
    q.off = block + placement_pad(block, q.start);
    q.admitted = true;
    S->active[q.client].push_back(Act{id, q.off, q.n, 0, q.start, q.fmt});
    ++S->n_admitted;
    return true;
}

// First come, first served; when the head waits for space (a large output
// and a fragmented arena), later requests of other clients may go first,
// each client's requests still in order (a client with a waiting request
// admits none after it), until the bytes admitted past the head reach half
// the arena: then admission waits for the head, so that it cannot starve.
void admit(Server *S)
{
    while (!S->pending.empty()) {
        if (S->pending.front().id != kGone) {
            if (!admit_one(S, S->pending.front().id))
                break;
            --S->n_pending;
            S->bypassed = 0;
        }
        S->pending.pop_front();
    }
    if (S->pending.empty() || S->bypassed >= S->arena->size() / 2 || !S->rescan)
        return;
    S->rescan = false;  // nothing can change until space is released or work queued
    S->held.assign(S->n_clients, 0);
    S->held[S->pending.front().client] = 1;
    size_t seen = 0;
    for (size_t k = 1; k < S->pending.size() && seen < kLookahead &&
                       S->bypassed < S->arena->size() / 2;
         ++k, ++seen) {
        Pend &q = S->pending[k];
        if (q.id == kGone)
            continue;
        if (!S->held[q.client] && block_bytes(q.n) <= S->arena->largest() &&
            admit_one(S, q.id)) {
            S->bypassed += block_bytes(q.n);
            q.id = kGone;
            --S->n_pending;
        } else {
            S->held[q.client] = 1;
        }
    }
}

// Rows per client in the next tick of `lane`: an equal share of the target
// tick for every busy client, at most chunk_rows (chunk_rows alone when no
// target is set).
uint64_t tick_rows(const Server *S, int lane)
{
    uint64_t rows = S->chunk_rows;
    if (S->tick_bytes) {
        uint64_t busy = 0;
        for (uint32_t c = lane; c < S->n_clients; c += kLanes)
            busy += !S->active[c].empty();
        const uint64_t share = busy ? S->tick_bytes / (busy * S->streams * 4) : rows;
        rows = std::max<uint64_t>(1, std::min<uint64_t>(rows, share));
    }
    return rows;
}

// Client c's piece of a tick of at most cap samples: its front request and
// the ones after it (run_piece).
RunPiece client_piece(Server *S, uint32_t c, uint64_t cap)
{
    const std::deque<Act> &act = S->active[c];
    S->run.clear();
    uint64_t have = 0;  // samples the collected requests still need
    for (size_t i = 0; i < act.size() && have < cap; ++i) {
        const Act &q = act[i];
        S->run.push_back(RunReq{q.off, q.n, q.done, q.fmt});
        have += q.n - q.done;
    }
    return run_piece(S->run.data(), S->run.size(), cap);
}

// a piece's window indices stay below 2^31 (format maps are 32-bit)
uint64_t piece_cap(const Server *S, uint64_t rows)
{
    return std::min<uint64_t>(rows * S->streams, 1ull << 31);
}

// Samples the next tick of `lane` would write.
uint64_t tick_samples(Server *S, int lane)
{
    const uint64_t cap = piece_cap(S, tick_rows(S, lane));
    uint64_t total = 0;
    for (uint32_t c = lane; c < S->n_clients; c += kLanes)
        if (!S->active[c].empty())
            total += client_piece(S, c, cap).m;
    return total;
}

// One tick of `lane`: one piece of every busy client of the lane, one launch
// on the lane's stream.
int launch_tick(Server *S, int lane)
{
    S->items.clear();
    S->item_map.clear();
    S->maps.clear();
    Tick tick;
    const uint64_t cap = piece_cap(S, tick_rows(S, lane));
    // clients lane, lane + kLanes, ... (none when the lane is past the last client)
    const uint32_t per_lane =
        (uint32_t)lane < S->n_clients ? (S->n_clients - lane + kLanes - 1) / kLanes : 0;
    for (uint32_t k = 0; k < per_lane; ++k) {
        const uint32_t c = lane + kLanes * ((S->rr[lane] + k) % per_lane);
        if (S->active[c].empty())
            continue;
        std::deque<Act> &act = S->active[c];
        const RunPiece pc = client_piece(S, c, cap);
        const Act &q0 = act.front();
        // the piece's output map: origin, then (start, format, shift) per
        // segment, then the end entry
        const uint64_t map_at = S->maps.size();
        const uintptr_t origin = reinterpret_cast<uintptr_t>(S->arena_base + pc.origin);
        S->maps.push_back((uint32_t)(origin & 0xFFFFFFFFu));
        S->maps.push_back((uint32_t)((uint64_t)origin >> 32));
        for (const Seg &g : pc.segs) {
            S->maps.push_back(g.b);
            S->maps.push_back((uint32_t)g.fmt);
            S->maps.push_back((uint32_t)((uint64_t)g.shift & 0xFFFFFFFFu));
            S->maps.push_back((uint32_t)((uint64_t)g.shift >> 32));
        }
        S->maps.insert(S->maps.end(), {kFmtEnd, 0u, 0u, 0u});
        const size_t first = S->items.size();
        piece_items(S->gens[c], S->streams, q0.start + q0.done, pc.m,
                    S->arena_base + pc.origin, RNG_U32, S->items);
        split_aligned(S->items, first);
        S->item_map.resize(S->items.size(), map_at);
        // the requests the piece completes, and how far it reaches into the last
        uint64_t left = pc.m;
        for (size_t j = 0; j < pc.touched; ++j) {
            Act &q = act.front();
            const uint64_t take = std::min(q.n - q.done, left);
            q.done += take;
            left -= take;
            if (q.done < q.n)
                break;
            tick.completing.push_back(q.id);
            act.pop_front();
        }
        S->samples += pc.m;
    }
    if (per_lane)
        S->rr[lane] = (S->rr[lane] + 1) % per_lane;
    if (S->items.empty())
        return RNG_OK;
    int st = RNG_OK;
    if (!S->plan[lane]) {
        S->plan[lane] = rng_plan_create(S->items.data(), S->items.size(), S->plan_threads,
                                        S->plan_ctas);
        st = S->plan[lane] ? RNG_OK : rng_last_error();
    }
    if (!st)
        st = plan_refill_mixed(S->plan[lane], S->items.data(), S->items.size(),
                               S->item_map.data(), S->maps.data(), S->maps.size(),
                               S->stream[lane]);
    if (!st)
        st = rng_plan_launch(S->plan[lane], S->stream[lane]);
    if (st)
        return st;
    if (S->spare_events.empty()) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess)
            return set_error(RNG_ERR_CUDA);
        S->spare_events.push_back(ev);
    }
    tick.ev = S->spare_events.back();
    S->spare_events.pop_back();
    st = cuda_status(cudaEventRecord(tick.ev, S->stream[lane]));
    if (st)
        return st;
    S->inflight[lane].push_back(std::move(tick));
    ++S->n_ticks;
    return RNG_OK;
}

bool lane_active(const Server *S, int lane)
{
    for (uint32_t c = lane; c < S->n_clients; c += kLanes)
        if (!S->active[c].empty())
            return true;
    return false;
}

bool has_active(const Server *S)
{
    for (int ln = 0; ln < kLanes; ++ln)
        if (lane_active(S, ln))
            return true;
    return false;
}

bool any_inflight(const Server *S)
{
    for (int ln = 0; ln < kLanes; ++ln)
        if (!S->inflight[ln].empty())
            return true;
    return false;
}

int progress(Server *S)
{
    int st = retire(S);
    if (st)
        return st;
    admit(S);
    for (int ln = 0; ln < kLanes; ++ln) {
        while ((int)S->inflight[ln].size() < kMaxInflight && lane_active(S, ln)) {
            // with a tick already running, wait for enough work to make the
            // next one worth a launch: a tick takes a client's whole adjacent
            // run, so one launched at once would often hold a few bytes
            if (!S->inflight[ln].empty() && S->tick_bytes &&
                4 * tick_samples(S, ln) < S->tick_bytes / 4)
                break;
            st = launch_tick(S, ln);
            if (st)
                return st;
        }
    }
    return RNG_OK;
}

void free_server(Server *S)
{
    if (!S)
        return;
    for (int ln = 0; ln < kLanes; ++ln)
        if (S->stream[ln])
            cudaStreamSynchronize(S->stream[ln]);
    for (int ln = 0; ln < kLanes; ++ln)
        rng_plan_destroy(S->plan[ln]);
    for (rng_handle h : S->gens)
        rng_destroy(h);
    for (int ln = 0; ln < kLanes; ++ln)
        for (auto &t : S->inflight[ln])
            cudaEventDestroy(t.ev);
    for (cudaEvent_t e : S->spare_events)
        cudaEventDestroy(e);
    if (S->t0)
        cudaEventDestroy(S->t0);
    for (int ln = 0; ln < kLanes; ++ln)
        if (S->stream[ln])
            cudaStreamDestroy(S->stream[ln]);
    cudaFree(S->arena_base);
    delete S->arena;
    delete S;
}

}  // namespace
}  // namespace gbrng

using namespace gbrng;

extern "C" rng_server_handle rng_server_create(int kind, uint32_t n_clients,
                                               uint64_t streams_per_client, uint64_t seed_base,
                                               uint64_t budget_bytes, uint32_t chunk_rows)
{
    if ((kind != RNG_MWC32 && kind != RNG_XOR128 && kind != RNG_KISS) || n_clients == 0 ||
        streams_per_client == 0 || chunk_rows == 0 || streams_per_client >= (1ull << 32)) {
        set_error(RNG_ERR_ARG);
        return nullptr;
    }
    const uint64_t per_stream = 4ull * words_of(kind) + (kind != RNG_XOR128 ? 4 : 0);
    const uint64_t state = per_stream * streams_per_client * n_clients;
    if (state + (1 << 20) > budget_bytes) {
        set_error(RNG_ERR_OOM);
        return nullptr;
    }
    Server *S = new (std::nothrow) Server();
    if (!S) {
        set_error(RNG_ERR_OOM);
        return nullptr;
    }
    S->kind = kind;
    S->n_clients = n_clients;
    S->streams = streams_per_client;
    S->chunk_rows = chunk_rows;
    cudaGetDevice(&S->device);
    S->active.resize(n_clients);
    S->cursor.assign(n_clients, 0);
    // Seeds 2^32 apart: stream s of client k starts splitmix64 at
    // seed_base + k * 2^32 + s, so no two streams of any clients share it.
    for (uint32_t k = 0; k < n_clients; ++k) {
        rng_handle h = rng_create(kind, streams_per_client, seed_base + ((uint64_t)k << 32));
        if (!h) {
            free_server(S);
            return nullptr;
        }
        S->gens.push_back(h);
    }
    const uint64_t arena = (budget_bytes - state) / kGranule * kGranule;
    int st = RNG_OK;
    if (cudaMalloc(&S->arena_base, arena) != cudaSuccess)
        st = set_error(RNG_ERR_OOM);
    if (!st)
        S->arena = new (std::nothrow) Arena(arena, kGranule);
    if (!st && !S->arena)
        st = set_error(RNG_ERR_OOM);
    for (int ln = 0; ln < kLanes && !st; ++ln)
        st = cuda_status(cudaStreamCreateWithFlags(&S->stream[ln], cudaStreamNonBlocking));
    if (!st)
        st = cuda_status(cudaEventCreate(&S->t0));
    if (!st)
        st = cuda_status(cudaEventRecord(S->t0, S->stream[0]));
    if (!st)
        st = cuda_status(cudaEventSynchronize(S->t0));
    for (uint32_t k = 0; k < n_clients && !st; ++k)
        st = rng_set_stream(S->gens[k], S->stream[k % kLanes]);
    if (st) {
        free_server(S);
        return nullptr;
    }
    return reinterpret_cast<rng_server_handle>(S);
}

extern "C" int rng_server_submit(rng_server_handle h, uint32_t client, uint64_t n_samples,
                                 int fmt, uint64_t *req_id)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S || client >= S->n_clients || n_samples == 0 || (fmt != RNG_U32 && fmt != RNG_F32) ||
        block_bytes(n_samples) > S->arena->size())
        return set_error(RNG_ERR_ARG);
    const uint64_t id = S->next_id++;
    Req q;
    q.client = client;
    q.n = n_samples;
    q.fmt = fmt;
    q.start = S->cursor[client];
    S->cursor[client] += n_samples;
    S->reqs.emplace(id, q);
    S->pending.push_back(Pend{id, n_samples, client});
    ++S->n_pending;
    S->rescan = true;
    if (req_id)
        *req_id = id;
    return RNG_OK;
}

extern "C" int rng_server_submit_many(rng_server_handle h, const uint32_t *clients,
                                      const uint64_t *n_samples, const int *fmts, size_t n,
                                      uint64_t *req_ids)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S || (n && (!clients || !n_samples || !fmts)))
        return set_error(RNG_ERR_ARG);
    for (size_t i = 0; i < n; ++i)  // all or nothing
        if (clients[i] >= S->n_clients || n_samples[i] == 0 ||
            (fmts[i] != RNG_U32 && fmts[i] != RNG_F32) ||
            block_bytes(n_samples[i]) > S->arena->size())
            return set_error(RNG_ERR_ARG);
    for (size_t i = 0; i < n; ++i) {
        int st = rng_server_submit(h, clients[i], n_samples[i], fmts[i], req_ids ? &req_ids[i]
                                                                            : nullptr);
        if (st)
            return st;
    }
    return RNG_OK;
}

extern "C" int rng_server_progress(rng_server_handle h)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S)
        return set_error(RNG_ERR_ARG);
    DeviceScope ds(S->device);
    int st = progress(S);
    return st ? st : (int)std::min<size_t>(S->done.size(), 0x7FFFFFFF);
}

extern "C" int rng_server_drain(rng_server_handle h)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S)
        return set_error(RNG_ERR_ARG);
    DeviceScope ds(S->device);
    for (;;) {
        int st = progress(S);
        if (st)
            return st;
        if (!any_inflight(S)) {
            if (S->n_pending == 0 && !has_active(S))
                return RNG_OK;
            if (!has_active(S))
                return set_error(RNG_ERR_BUSY);  // waiting requests need released space
            continue;
        }
        for (int ln = 0; ln < kLanes; ++ln) {
            if (S->inflight[ln].empty())
                continue;
            cudaError_t e = cudaEventSynchronize(S->inflight[ln].front().ev);
            if (e != cudaSuccess)
                return cuda_status(e);
            break;
        }
    }
}

extern "C" int rng_server_take(rng_server_handle h, uint64_t *ids, double *done_ms, int cap)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S || cap < 0 || (cap > 0 && !ids))
        return set_error(RNG_ERR_ARG);
    int n = 0;
    while (n < cap && !S->done.empty()) {
        ids[n] = S->done.front().first;
        if (done_ms)
            done_ms[n] = S->done.front().second;
        S->done.pop_front();
        ++n;
    }
    return n;
}

extern "C" int rng_server_result(rng_server_handle h, uint64_t req_id, void **dev_ptr,
                                 uint64_t *n_samples, int *fmt, uint32_t *client, uint64_t *start)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S)
        return set_error(RNG_ERR_ARG);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end() || !it->second.completed)
        return set_error(RNG_ERR_ARG);
    const Req &q = it->second;
    if (dev_ptr)
        *dev_ptr = S->arena_base + q.off / 4;
    if (n_samples)
        *n_samples = q.n;
    if (fmt)
        *fmt = q.fmt;
    if (client)
        *client = q.client;
    if (start)
        *start = q.start;
    return RNG_OK;
}

extern "C" int rng_server_copy(rng_server_handle h, uint64_t req_id, void *dst,
                               uint64_t offset, uint64_t count, void *cuda_stream)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S || !dst)
        return set_error(RNG_ERR_ARG);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end() || !it->second.completed || offset > it->second.n ||
        count > it->second.n - offset)
        return set_error(RNG_ERR_ARG);
    if (count == 0)
        return RNG_OK;
    DeviceScope ds(S->device);
    // a completed request's tick has finished: any stream may copy it
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const uint32_t *src = S->arena_base + it->second.off / 4 + offset;
    return cuda_status(cudaMemcpyAsync(dst, src, count * 4, cudaMemcpyDefault, st));
}

extern "C" int rng_server_release(rng_server_handle h, uint64_t req_id)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S)
        return set_error(RNG_ERR_ARG);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end() || !it->second.completed)
        return set_error(RNG_ERR_ARG);
    S->arena->release(it->second.block, block_bytes(it->second.n));
    S->rescan = true;
    S->reqs.erase(it);
    return RNG_OK;
}

extern "C" int rng_server_release_many(rng_server_handle h, const uint64_t *req_ids, size_t n)
{
    if (n && !req_ids)
        return set_error(RNG_ERR_ARG);
    int st = RNG_OK;
    for (size_t i = 0; i < n; ++i) {
        int e = rng_server_release(h, req_ids[i]);
        if (e && !st)
            st = e;
    }
    return st;
}

extern "C" int rng_server_stats(rng_server_handle h, uint64_t *out8)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S || !out8)
        return set_error(RNG_ERR_ARG);
    out8[0] = S->next_id;
    out8[1] = S->n_admitted;
    out8[2] = S->n_completed;
    out8[3] = S->n_ticks;
    out8[4] = S->samples;
    out8[5] = S->arena->used();
    out8[6] = S->arena->size();
    out8[7] = S->n_pending;
    return RNG_OK;
}

extern "C" int rng_server_set_tick_bytes(rng_server_handle h, uint64_t bytes)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S)
        return set_error(RNG_ERR_ARG);
    S->tick_bytes = bytes;
    return RNG_OK;
}

extern "C" int rng_server_set_plan_shape(rng_server_handle h, int threads, int ctas_per_sm)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S || threads < 32 || threads > 512 || (threads & (threads - 1)) || ctas_per_sm < 0 ||
        ctas_per_sm > 32)
        return set_error(RNG_ERR_ARG);
    DeviceScope ds(S->device);
    // the lanes' plans are rebuilt with the new shape at their next tick;
    // wait for the ticks that still read them
    for (int ln = 0; ln < kLanes; ++ln) {
        if (!S->plan[ln])
            continue;
        int st = cuda_status(cudaStreamSynchronize(S->stream[ln]));
        if (st)
            return st;
        rng_plan_destroy(S->plan[ln]);
        S->plan[ln] = nullptr;
    }
    S->plan_threads = threads;
    S->plan_ctas = ctas_per_sm;
    return RNG_OK;
}

extern "C" void rng_server_destroy(rng_server_handle h)
{
    Server *S = reinterpret_cast<Server *>(h);
    if (!S)
        return;
    DeviceScope ds(S->device);
    free_server(S);
}
