// Serving: a continuous-batching request loop over resident activation caches.
//
// Markov chains of different lengths N register their current configuration; a
// request carries single-flip proposals for one chain and receives their
// log-amplitude ratios (Sec. "ABACUS": the ratios a Metropolis step or a local
// energy needs, served from the chain's cache).  One worker thread per server
//  * takes every pending request that fits the next batch (requests that arrive
//    while earlier batches are on the GPU join the next one),
//  * admits the chains of the batch against a device-memory budget: a chain
//    without a resident cache gets one built (dysonnet_forward_cache), evicting
//    the least recently used idle caches when the budget would be exceeded,
//  * launches the whole batch as one kernel over several caches (k_abacus_multi,
//    one CTA per flip) on one of two streams, so that batch k+1 is formed and
//    launched while batch k is still running,
//  * copies results to the callers' host buffers and timestamps completion.
// The recompute mode serves the same requests by full forward passes of every
// proposal (dn_recompute_flip_ratios), the baseline the caches replace.
//
// The persistent mode keeps one kernel resident instead of launching one per batch: the
// worker appends each admitted request's proposals to a work queue in host-mapped memory
// and publishes them by advancing a counter; the CTAs of k_abacus_serve claim items as
// they appear, run the flip-list body on the item's cache and hand the ratio back through
// the same mapped memory.  Requests arriving while others are on the GPU are appended
// behind them with no launch in between.  The kernel waits for work only up to an idle
// limit, then leaves with DN_ETIMEOUT in its status word (dn_server_kernel_status); the
// worker launches it again when work arrives, and stops it before a new chain's cache is
// built so that the build's kernels get the SMs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dn_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    unsigned long long ticket = 0, item0 = 0;
    int chain = 0, F = 0;
    std::vector<int32_t> sites;   // [F][2]
    double *out_host = nullptr;
    Clock::time_point t_submit, t_done;
    dn_status status = DN_OK;
    bool done = false;
};

struct Chain {
    int N = 0;
    int8_t *spins_dev = nullptr;
    dn_cache *cache = nullptr;
    size_t bytes = 0;
    unsigned long long last_use = 0;
    int in_flight = 0;   // batches on the GPU that use this chain
    int slot = -1;       // persistent mode: row of the device descriptor table
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int32_t *h_i = nullptr, *d_i = nullptr;   // [sites 2F | sample F | cache_of F]
    double *h_out = nullptr, *d_out = nullptr;
    unsigned char *h_desc = nullptr, *d_desc = nullptr;
    size_t bytes_i = 0, bytes_out = 0, bytes_desc = 0;
    std::vector<Request *> reqs;
    std::vector<int> offs, chains;
    bool busy = false;
};

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

}  // namespace

struct dn_server {
    dn_model *m = nullptr;
    int prec = DN_FP32, mode = DN_SERVE_ABACUS, device = 0, max_flips = 0, max_chains = 0;
    size_t budget = 0, desc_bytes = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<unsigned long long, Request *> reqs;
    std::unordered_map<int, Chain> chains;
    size_t resident = 0;
    unsigned long long next_ticket = 1, clock = 0;
    bool stop = false;
    std::thread worker;
    Slot slots[2];
    dn_server_stats stats{};
    cudaStream_t setup = nullptr;
    // persistent mode
    bool persistent = false;
    dn::ServeQueue *q = nullptr, *q_dev = nullptr;         // host-mapped
    dn::ServeItems items{}, items_dev{};                   // host-mapped ring of cap items
    unsigned long long *ctl_dev = nullptr;                  // ticket counter, closing word (device)
    unsigned char *desc_tab = nullptr;                      // [kDescSlots] descriptors (device)
    std::vector<int> free_slots;
    unsigned long long next_item = 0, done_upto = 0;
    cudaStream_t kst = nullptr;
    cudaEvent_t kev = nullptr;
    bool k_launched = false;
    long long idle_ns = 200000000;                          // 0.2 s
    int ctas = 0;
    std::mutex kmu;                                         // kernel launch and status
};

namespace {

constexpr int kDescSlots = 1024;   // resident caches addressable by the persistent kernel

bool fp64(const dn_server *s) { return s->prec == DN_FP64; }

// Drop the cache of chain c (its batches must be done).
void drop_cache(dn_server *s, Chain &c) {
    if (c.cache) {
        dn_cache_destroy(c.cache);
        c.cache = nullptr;
        s->resident -= c.bytes;
        c.bytes = 0;
    }
    if (c.slot >= 0) {
        s->free_slots.push_back(c.slot);
        c.slot = -1;
    }
}

// Persistent kernel: is it running (launched and not finished)?  Called with kmu held.
bool kernel_running(dn_server *s) {
    if (!s->k_launched) return false;
    const cudaError_t e = cudaEventQuery(s->kev);
    if (e == cudaErrorNotReady) return true;
    if (e != cudaSuccess) cudaGetLastError();
    return false;
}

// Ask the persistent kernel to leave and wait for it (it finishes the items already
// published first); the wait on the host is bounded by 30 s.
void stop_kernel(dn_server *s) {
    std::lock_guard<std::mutex> lk(s->kmu);
    if (!s->k_launched) return;
    *((volatile unsigned int *)&s->q->stop) = 1u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    const auto t0 = Clock::now();
    while (kernel_running(s) && seconds(Clock::now() - t0) < 30.0) std::this_thread::sleep_for(std::chrono::microseconds(50));
    if (!kernel_running(s)) s->k_launched = false;
    *((volatile unsigned int *)&s->q->stop) = 0u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
}

// Launch the persistent kernel if items are outstanding and it is not running.  Called
// by the worker only (it alone publishes items).  The new launch's tickets start at the
// first item not yet served; the kernel drops those after it that the previous launch
// served (their state words say so).
dn_status ensure_kernel(dn_server *s) {
    std::lock_guard<std::mutex> lk(s->kmu);
    if (kernel_running(s)) return DN_OK;
    s->k_launched = false;
    *((volatile int *)&s->q->status) = DN_OK;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    const unsigned long long cap = (unsigned long long)s->items.cap;
    unsigned long long base = s->done_upto;
    while (base < s->next_item && *((volatile unsigned long long *)&s->items.done[base % cap]) == 2 * base + 2) ++base;
    const int WF = 2 * s->m->desc.w + 1;
    cudaError_t e = cudaMemsetAsync(s->ctl_dev, 0, 2 * sizeof(unsigned long long), s->kst);
    if (e == cudaSuccess)
        e = fp64(s) ? dn::launch_abacus_serve<double>(s->m, WF, s->desc_tab, s->q_dev, s->items_dev, s->ctl_dev, base,
                                                      s->idle_ns, s->ctas, s->kst)
                    : dn::launch_abacus_serve<float>(s->m, WF, s->desc_tab, s->q_dev, s->items_dev, s->ctl_dev, base,
                                                     s->idle_ns, s->ctas, s->kst);
    if (e == cudaSuccess) e = cudaEventRecord(s->kev, s->kst);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DN_ECUDA;
    }
    s->k_launched = true;
    return DN_OK;
}

// Make room for `need` bytes by evicting idle caches, least recently used first.
// `keep` lists the chains of the batch being formed.  Called with s->mu held.
bool make_room(dn_server *s, size_t need, const std::vector<int> &keep) {
    while (s->resident + need > s->budget) {
        Chain *victim = nullptr;
        for (auto &kv : s->chains) {
            Chain &c = kv.second;
            if (!c.cache || c.in_flight > 0) continue;
            if (std::find(keep.begin(), keep.end(), kv.first) != keep.end()) continue;
            if (!victim || c.last_use < victim->last_use) victim = &c;
        }
        if (!victim) return false;
        drop_cache(s, *victim);
        s->stats.evictions++;
    }
    return true;
}

// Build chain c's cache on stream st and wait for it: later batches may run on the
// other stream, which nothing orders after this one.
dn_status build_cache(dn_server *s, Chain &c, cudaStream_t st) {
    dn_cache *cache = nullptr;
    dn_status r = dysonnet_forward_cache(s->m, c.N, c.spins_dev, 1, (dn_precision)s->prec, 1, st, &cache, nullptr);
    if (r != DN_OK) return r;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        dn_cache_destroy(cache);
        return DN_ECUDA;
    }
    c.cache = cache;
    c.bytes = dn_cache_bytes(s->m, c.N, 1, (dn_precision)s->prec, 1);
    s->resident += c.bytes;
    s->stats.cache_builds++;
    return DN_OK;
}

void finish(dn_server *s, Slot &sl, dn_status status) {
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t k = 0; k < sl.reqs.size(); ++k) {
        Request *r = sl.reqs[k];
        if (status == DN_OK) memcpy(r->out_host, sl.h_out + sl.offs[k], (size_t)r->F * sizeof(double));
        r->status = status;
        r->t_done = now;
        r->done = true;
    }
    for (int c : sl.chains) s->chains[c].in_flight--;
    s->stats.batches++;
    sl.reqs.clear();
    sl.offs.clear();
    sl.chains.clear();
    sl.busy = false;
    s->cv_done.notify_all();
}

// Form and launch one batch on slot sl: 0 when nothing could be admitted, 1 when a
// batch is in flight on sl, 2 when it failed (its requests are already completed).
int launch_batch(dn_server *s, Slot &sl) {
    std::vector<Request *> batch;
    std::vector<int> bchains;
    int flips = 0;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        while (!s->pending.empty()) {
            Request *r = s->pending.front();
            if (flips + r->F > s->max_flips && !batch.empty()) break;
            const bool new_chain = std::find(bchains.begin(), bchains.end(), r->chain) == bchains.end();
            if (new_chain && (int)bchains.size() >= s->max_chains) break;
            Chain &c = s->chains[r->chain];
            if (new_chain && s->mode == DN_SERVE_ABACUS && !c.cache) {
                const size_t need = dn_cache_bytes(s->m, c.N, 1, (dn_precision)s->prec, 1);
                if (!make_room(s, need, bchains)) break;   // wait until in-flight batches release caches
                dn_status b = build_cache(s, c, sl.st);
                if (b != DN_OK) {
                    s->pending.pop_front();
                    r->status = b;
                    r->t_done = Clock::now();
                    r->done = true;
                    s->cv_done.notify_all();
                    continue;
                }
            }
            s->pending.pop_front();
            if (new_chain) {
                bchains.push_back(r->chain);
                c.in_flight++;
            }
            c.last_use = ++s->clock;
            batch.push_back(r);
            flips += r->F;
        }
    }
    if (batch.empty()) return 0;
    // Stage the batch: sites, sample 0 (every cache holds one configuration), cache index.
    int32_t *h_sites = sl.h_i, *h_sample = sl.h_i + 2 * s->max_flips, *h_cof = h_sample + s->max_flips;
    int off = 0;
    for (Request *r : batch) {
        const int ci = (int)(std::find(bchains.begin(), bchains.end(), r->chain) - bchains.begin());
        memcpy(h_sites + 2 * off, r->sites.data(), (size_t)r->F * 2 * sizeof(int32_t));
        for (int f = 0; f < r->F; ++f) {
            h_sample[off + f] = 0;
            h_cof[off + f] = ci;
        }
        sl.offs.push_back(off);
        off += r->F;
    }
    sl.reqs = batch;
    sl.chains = bchains;
    sl.busy = true;
    int32_t *d_sites = sl.d_i, *d_sample = sl.d_i + 2 * s->max_flips, *d_cof = d_sample + s->max_flips;
    cudaError_t e = cudaMemcpyAsync(d_sites, h_sites, (size_t)off * 2 * sizeof(int32_t), cudaMemcpyHostToDevice, sl.st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_sample, h_sample, (size_t)off * sizeof(int32_t), cudaMemcpyHostToDevice, sl.st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cof, h_cof, (size_t)off * sizeof(int32_t), cudaMemcpyHostToDevice, sl.st);
    if (e == cudaSuccess && s->mode == DN_SERVE_ABACUS) {
        for (size_t k = 0; k < bchains.size(); ++k) {
            Chain &c = s->chains[bchains[k]];
            if (fp64(s))
                dn::abacus_desc<double>(s->m, s->m->plan64.at(c.N), s->m->w64, c.cache, sl.h_desc + k * s->desc_bytes);
            else
                dn::abacus_desc<float>(s->m, s->m->plan32.at(c.N), s->m->w32, c.cache, sl.h_desc + k * s->desc_bytes);
        }
        e = cudaMemcpyAsync(sl.d_desc, sl.h_desc, bchains.size() * s->desc_bytes, cudaMemcpyHostToDevice, sl.st);
        const int WF = 2 * s->m->desc.w + 1;
        if (e == cudaSuccess)
            e = fp64(s) ? dn::launch_abacus_multi<double>(s->m, WF, sl.d_desc, d_cof, d_sample, d_sites, off, sl.d_out,
                                                          sl.st)
                        : dn::launch_abacus_multi<float>(s->m, WF, sl.d_desc, d_cof, d_sample, d_sites, off, sl.d_out,
                                                         sl.st);
    } else if (e == cudaSuccess) {
        // Recompute: every proposal of a request by full forward passes of its chain.
        for (size_t k = 0; k < batch.size() && e == cudaSuccess; ++k) {
            Request *r = batch[k];
            Chain &c = s->chains[r->chain];
            dn_status st = dn_recompute_flip_ratios(s->m, c.N, c.spins_dev, 1, d_sample + sl.offs[k],
                                                    d_sites + 2 * sl.offs[k], r->F, (dn_precision)s->prec, sl.st,
                                                    sl.d_out + sl.offs[k]);
            if (st != DN_OK) e = cudaErrorUnknown;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)off * sizeof(double), cudaMemcpyDeviceToHost, sl.st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.st);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.flips += off;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(sl.st);
        finish(s, sl, DN_ECUDA);
        return 2;
    }
    return 1;
}

void worker_main(dn_server *s) {
    cudaSetDevice(s->device);
    std::deque<int> inflight;   // busy slots in launch order
    for (;;) {
        bool have_pending, stopping;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (inflight.empty()) s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            have_pending = !s->pending.empty();
            stopping = s->stop;
        }
        if (stopping && !have_pending && inflight.empty()) break;
        int launched = 0;
        if (have_pending && inflight.size() < 2) {
            const int k = s->slots[0].busy ? 1 : 0;
            launched = launch_batch(s, s->slots[k]);
            if (launched == 1) inflight.push_back(k);
        }
        if (!inflight.empty()) {
            // Complete the oldest batch; block on it only when both slots are busy or there is
            // nothing else to do.
            Slot &o = s->slots[inflight.front()];
            const bool block = inflight.size() == 2 || (!launched && !have_pending);
            const cudaError_t q = block ? cudaEventSynchronize(o.ev) : cudaEventQuery(o.ev);
            if (q != cudaErrorNotReady) {
                if (q != cudaSuccess) cudaGetLastError();
                finish(s, o, q == cudaSuccess ? DN_OK : DN_ECUDA);
                inflight.pop_front();
            } else if (!launched) {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        } else if (have_pending && !launched) {
            // Nothing admissible with nothing in flight: the budget cannot hold the next chain.
            std::lock_guard<std::mutex> lk(s->mu);
            Request *r = s->pending.front();
            s->pending.pop_front();
            r->status = DN_ENOMEM;
            r->t_done = Clock::now();
            r->done = true;
            s->cv_done.notify_all();
        }
    }
}

// Persistent mode: give chain c a row of the descriptor table holding its cache's
// descriptor (written and synchronised before any item refers to it).
dn_status bind_slot(dn_server *s, Chain &c) {
    if (c.slot >= 0) return DN_OK;
    if (s->free_slots.empty()) return DN_ENOMEM;
    const int slot = s->free_slots.back();
    std::vector<unsigned char> d(s->desc_bytes);
    if (fp64(s)) dn::abacus_desc<double>(s->m, s->m->plan64.at(c.N), s->m->w64, c.cache, d.data());
    else dn::abacus_desc<float>(s->m, s->m->plan32.at(c.N), s->m->w32, c.cache, d.data());
    if (cudaMemcpyAsync(s->desc_tab + (size_t)slot * s->desc_bytes, d.data(), s->desc_bytes, cudaMemcpyHostToDevice,
                        s->setup) != cudaSuccess ||
        cudaStreamSynchronize(s->setup) != cudaSuccess) {
        cudaGetLastError();
        return DN_ECUDA;
    }
    s->free_slots.pop_back();
    c.slot = slot;
    return DN_OK;
}

void fail_request(dn_server *s, Request *r, dn_status st) {
    r->status = st;
    r->t_done = Clock::now();
    r->done = true;
    s->cv_done.notify_all();
}

void worker_persistent(dn_server *s) {
    cudaSetDevice(s->device);
    std::deque<Request *> inflight;   // requests whose items are published, in publication order
    const unsigned long long cap = (unsigned long long)s->items.cap;
    for (;;) {
        bool stopping;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (inflight.empty())
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->stop || !s->pending.empty(); });
            stopping = s->stop && s->pending.empty() && inflight.empty();
        }
        if (stopping) break;
        bool progress = false;
        // Publish every pending request whose proposals fit in the ring, admitting its chain.
        for (;;) {
            Request *r = nullptr;
            Chain *c = nullptr;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->pending.empty()) break;
                r = s->pending.front();
                if (s->next_item + (unsigned long long)r->F - s->done_upto > cap) break;   // ring full: wait
                c = &s->chains[r->chain];
                if (!c->cache) {
                    const size_t need = dn_cache_bytes(s->m, c->N, 1, (dn_precision)s->prec, 1);
                    if (!make_room(s, need, {r->chain})) {
                        if (!inflight.empty()) break;   // wait until in-flight requests release caches
                        s->pending.pop_front();
                        fail_request(s, r, DN_ENOMEM);
                        continue;
                    }
                    stop_kernel(s);                     // the build's kernels need the SMs
                    const dn_status b = build_cache(s, *c, s->setup);
                    if (b != DN_OK) {
                        s->pending.pop_front();
                        fail_request(s, r, b);
                        continue;
                    }
                }
                const dn_status bs = bind_slot(s, *c);
                if (bs != DN_OK) {
                    s->pending.pop_front();
                    fail_request(s, r, bs);
                    continue;
                }
                s->pending.pop_front();
                c->in_flight++;
                c->last_use = ++s->clock;
                s->stats.flips += r->F;
                s->stats.batches++;
            }
            // The ring slots of items next_item .. next_item + F - 1 are free (done_upto).
            for (int f = 0; f < r->F; ++f) {
                const unsigned long long i = s->next_item + f;
                const int slot = (int)(i % cap);
                s->items.cache[slot] = c->slot;
                s->items.sites[2 * slot] = r->sites[2 * f];
                s->items.sites[2 * slot + 1] = r->sites[2 * f + 1];
                s->items.done[slot] = 2 * i + 1;   // published
            }
            r->item0 = s->next_item;
            s->next_item += (unsigned long long)r->F;
            std::atomic_thread_fence(std::memory_order_release);
            *((volatile unsigned long long *)&s->q->tail) = s->next_item;
            std::atomic_thread_fence(std::memory_order_seq_cst);
            inflight.push_back(r);
            progress = true;
        }
        if (!inflight.empty() && ensure_kernel(s) != DN_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            for (Request *r : inflight) {
                s->chains[r->chain].in_flight--;
                fail_request(s, r, DN_ECUDA);
            }
            inflight.clear();
            s->done_upto = s->next_item;
        }
        // Complete requests in publication order (ring slots are released in that order).
        while (!inflight.empty()) {
            Request *r = inflight.front();
            bool all = true;
            for (int f = 0; f < r->F && all; ++f) {
                const unsigned long long i = r->item0 + f;
                all = *((volatile unsigned long long *)&s->items.done[i % cap]) == 2 * i + 2;
            }
            if (!all) break;
            std::atomic_thread_fence(std::memory_order_acquire);
            for (int f = 0; f < r->F; ++f) r->out_host[f] = ((volatile double *)s->items.out)[(r->item0 + f) % cap];
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->chains[r->chain].in_flight--;
                r->status = DN_OK;
                r->t_done = Clock::now();
                r->done = true;
                s->cv_done.notify_all();
            }
            s->done_upto = r->item0 + (unsigned long long)r->F;
            inflight.pop_front();
            progress = true;
        }
        if (!progress && !inflight.empty()) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    stop_kernel(s);
}

void free_slot(Slot &sl) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.h_i) cudaFreeHost(sl.h_i);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    if (sl.h_desc) cudaFreeHost(sl.h_desc);
    if (sl.d_i) dn::dev_free(sl.d_i, sl.bytes_i, sl.st);
    if (sl.d_out) dn::dev_free(sl.d_out, sl.bytes_out, sl.st);
    if (sl.d_desc) dn::dev_free(sl.d_desc, sl.bytes_desc, sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.st) {
        cudaStreamSynchronize(sl.st);
        cudaStreamDestroy(sl.st);
    }
    sl = Slot{};
}

void destroy_server(dn_server *s) {
    for (auto &sl : s->slots) free_slot(sl);
    if (s->kst) {
        cudaStreamSynchronize(s->kst);
        cudaStreamDestroy(s->kst);
    }
    if (s->kev) cudaEventDestroy(s->kev);
    if (s->q) cudaFreeHost(s->q);
    if (s->items.cache) cudaFreeHost(s->items.cache);
    if (s->items.sites) cudaFreeHost(s->items.sites);
    if (s->items.out) cudaFreeHost(s->items.out);
    if (s->items.done) cudaFreeHost(s->items.done);
    if (s->ctl_dev) cudaFree(s->ctl_dev);
    if (s->desc_tab) cudaFree(s->desc_tab);
    for (auto &kv : s->chains) {
        drop_cache(s, kv.second);
        if (kv.second.spins_dev) dn::dev_free(kv.second.spins_dev, (size_t)kv.second.N, s->setup);
    }
    for (auto &kv : s->reqs) delete kv.second;
    if (s->setup) {
        cudaStreamSynchronize(s->setup);
        cudaStreamDestroy(s->setup);
    }
    delete s;
}

}  // namespace

extern "C" {

dn_status dn_server_create(dn_model *m, dn_precision prec, int mode, size_t hbm_budget_bytes, int max_batch_flips,
                           int max_batch_chains, dn_server **out) {
    if (!out) return DN_EINVAL;
    *out = nullptr;
    if (!m || (prec != DN_FP64 && prec != DN_FP32 && prec != DN_BF16) ||
        (mode != DN_SERVE_ABACUS && mode != DN_SERVE_RECOMPUTE && mode != DN_SERVE_PERSISTENT) ||
        max_batch_flips < 1 || max_batch_chains < 1)
        return DN_EINVAL;
    dn_server *s = new dn_server();
    s->m = m;
    s->prec = prec;
    s->mode = mode;
    s->budget = hbm_budget_bytes;
    s->max_flips = max_batch_flips;
    s->max_chains = max_batch_chains;
    s->desc_bytes =
        ((prec == DN_FP64 ? dn::abacus_desc_bytes<double>() : dn::abacus_desc_bytes<float>()) + 15) & ~(size_t)15;
    cudaGetDevice(&s->device);
    bool ok = cudaStreamCreateWithFlags(&s->setup, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &sl : s->slots) {
        if (!ok) break;
        sl.bytes_i = (size_t)4 * max_batch_flips * sizeof(int32_t);
        sl.bytes_out = (size_t)max_batch_flips * sizeof(double);
        sl.bytes_desc = (size_t)max_batch_chains * s->desc_bytes;
        ok = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaMallocHost(&sl.h_i, sl.bytes_i) == cudaSuccess && cudaMallocHost(&sl.h_out, sl.bytes_out) == cudaSuccess &&
             cudaMallocHost(&sl.h_desc, sl.bytes_desc) == cudaSuccess;
        if (!ok) break;
        sl.d_i = static_cast<int32_t *>(dn::dev_alloc(sl.bytes_i, sl.st));
        sl.d_out = static_cast<double *>(dn::dev_alloc(sl.bytes_out, sl.st));
        sl.d_desc = static_cast<unsigned char *>(dn::dev_alloc(sl.bytes_desc, sl.st));
        ok = sl.d_i && sl.d_out && sl.d_desc;
    }
    if (ok && mode == DN_SERVE_PERSISTENT) {
        // Work queue and ring in host-mapped memory (read by the kernel while it runs), the
        // ticket counter, the closing word and the descriptor table in device memory.
        s->persistent = true;
        const int cap = 4 * max_batch_flips;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        s->ctas = 2 * (sms > 0 ? sms : 1);
        void *hq = nullptr, *hc = nullptr, *hs = nullptr, *ho = nullptr, *hd = nullptr;
        ok = cudaHostAlloc(&hq, sizeof(dn::ServeQueue), cudaHostAllocMapped) == cudaSuccess &&
             cudaHostAlloc(&hc, (size_t)cap * sizeof(int32_t), cudaHostAllocMapped) == cudaSuccess &&
             cudaHostAlloc(&hs, (size_t)cap * 2 * sizeof(int32_t), cudaHostAllocMapped) == cudaSuccess &&
             cudaHostAlloc(&ho, (size_t)cap * sizeof(double), cudaHostAllocMapped) == cudaSuccess &&
             cudaHostAlloc(&hd, (size_t)cap * sizeof(unsigned long long), cudaHostAllocMapped) == cudaSuccess;
        s->q = static_cast<dn::ServeQueue *>(hq);
        s->items = dn::ServeItems{static_cast<int32_t *>(hc), static_cast<int32_t *>(hs), static_cast<double *>(ho),
                                  static_cast<unsigned long long *>(hd), cap};
        if (ok) {
            memset(hq, 0, sizeof(dn::ServeQueue));
            memset(hd, 0, (size_t)cap * sizeof(unsigned long long));
            void *dq = nullptr, *dc = nullptr, *ds = nullptr, *dout = nullptr, *dd = nullptr;
            ok = cudaHostGetDevicePointer(&dq, hq, 0) == cudaSuccess && cudaHostGetDevicePointer(&dc, hc, 0) == cudaSuccess &&
                 cudaHostGetDevicePointer(&ds, hs, 0) == cudaSuccess && cudaHostGetDevicePointer(&dout, ho, 0) == cudaSuccess &&
                 cudaHostGetDevicePointer(&dd, hd, 0) == cudaSuccess;
            s->q_dev = static_cast<dn::ServeQueue *>(dq);
            s->items_dev = dn::ServeItems{static_cast<int32_t *>(dc), static_cast<int32_t *>(ds),
                                          static_cast<double *>(dout), static_cast<unsigned long long *>(dd), cap};
        }
        ok = ok && cudaMalloc(&s->ctl_dev, 2 * sizeof(unsigned long long)) == cudaSuccess &&
             cudaMemset(s->ctl_dev, 0, 2 * sizeof(unsigned long long)) == cudaSuccess &&
             cudaMalloc(&s->desc_tab, (size_t)kDescSlots * s->desc_bytes) == cudaSuccess &&
             cudaStreamCreateWithFlags(&s->kst, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->kev, cudaEventDisableTiming) == cudaSuccess &&
             cudaDeviceSynchronize() == cudaSuccess;
        for (int k = kDescSlots - 1; k >= 0; --k) s->free_slots.push_back(k);
    }
    if (!ok) {
        cudaGetLastError();
        destroy_server(s);
        return DN_ENOMEM;
    }
    s->worker = std::thread(s->persistent ? worker_persistent : worker_main, s);
    *out = s;
    return DN_OK;
}

dn_status dn_server_set_chain(dn_server *s, int chain, int N, const int8_t *spins_host, int build_now) {
    if (!s || chain < 0 || N < 1 || !spins_host) return DN_EINVAL;
    for (int i = 0; i < N; ++i)
        if (spins_host[i] != 1 && spins_host[i] != -1) return DN_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    Chain &c = s->chains[chain];
    if (c.in_flight > 0) return DN_EINVAL;
    for (Request *r : s->pending)
        if (r->chain == chain) return DN_EINVAL;
    drop_cache(s, c);
    if (c.spins_dev && c.N != N) {
        dn::dev_free(c.spins_dev, (size_t)c.N, s->setup);
        c.spins_dev = nullptr;
    }
    c.N = N;
    if (!c.spins_dev) c.spins_dev = static_cast<int8_t *>(dn::dev_alloc((size_t)N, s->setup));
    if (!c.spins_dev) return DN_ENOMEM;
    if (cudaMemcpyAsync(c.spins_dev, spins_host, (size_t)N, cudaMemcpyHostToDevice, s->setup) != cudaSuccess ||
        cudaStreamSynchronize(s->setup) != cudaSuccess) {
        cudaGetLastError();
        return DN_ECUDA;
    }
    if (build_now && s->mode != DN_SERVE_RECOMPUTE) {
        if (!make_room(s, dn_cache_bytes(s->m, N, 1, (dn_precision)s->prec, 1), {chain})) return DN_ENOMEM;
        if (s->persistent) stop_kernel(s);   // the build's kernels need the SMs
        dn_status r = build_cache(s, c, s->setup);
        if (r != DN_OK) return r;
        if (cudaStreamSynchronize(s->setup) != cudaSuccess) {
            cudaGetLastError();
            return DN_ECUDA;
        }
        c.last_use = ++s->clock;
    }
    return DN_OK;
}

dn_status dn_server_submit(dn_server *s, int chain, const int32_t *sites_host, int F, double *out_host,
                           unsigned long long *ticket) {
    if (!s || !sites_host || !out_host || !ticket || F < 1 || F > s->max_flips) return DN_EINVAL;
    Request *r = new Request();
    r->chain = chain;
    r->F = F;
    r->sites.assign(sites_host, sites_host + 2 * (size_t)F);
    r->out_host = out_host;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->chains.find(chain);
        if (it == s->chains.end() || !it->second.spins_dev) {
            delete r;
            return DN_EINVAL;
        }
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->reqs[r->ticket] = r;
        s->pending.push_back(r);
        s->stats.requests++;
    }
    s->cv_work.notify_one();
    return DN_OK;
}

dn_status dn_server_wait(dn_server *s, unsigned long long ticket, double timeout_s, double *latency_s) {
    if (!s) return DN_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return DN_EINVAL;
    Request *r = it->second;
    const auto dl = std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s);
    if (!s->cv_done.wait_for(lk, dl, [&] { return r->done; })) return DN_ETIMEOUT;
    if (latency_s) *latency_s = seconds(r->t_done - r->t_submit);
    const dn_status st = r->status;
    s->reqs.erase(it);
    delete r;
    return st;
}

dn_status dn_server_set_idle_limit(dn_server *s, double seconds_) {
    if (!s || !s->persistent || !(seconds_ > 0.0) || seconds_ > 3600.0) return DN_EINVAL;
    std::lock_guard<std::mutex> lk(s->kmu);
    s->idle_ns = (long long)(seconds_ * 1e9);
    return DN_OK;
}

dn_status dn_server_kernel_status(dn_server *s, double wait_s, int *running) {
    if (!s || !s->persistent) return DN_EINVAL;
    const auto t0 = Clock::now();
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->kmu);
            const bool run = kernel_running(s);
            if (!run || seconds(Clock::now() - t0) >= wait_s) {
                if (running) *running = run ? 1 : 0;
                if (run) return DN_OK;
                std::atomic_thread_fence(std::memory_order_acquire);
                return (dn_status) * ((volatile int *)&s->q->status);
            }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

dn_status dn_server_get_stats(dn_server *s, dn_server_stats *out) {
    if (!s || !out) return DN_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->resident_bytes = s->resident;
    return DN_OK;
}

void dn_server_destroy(dn_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    destroy_server(s);
}

}  // extern "C"
