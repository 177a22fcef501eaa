// serve.cu -- canny_serve: a continuous-batching request loop over the batch API.
//
// Requests (host images with arrival times) are admitted in arrival order as
// device memory frees up: each admitted request gets its input and output
// buffers from a device arena of a fixed byte budget, and the idle streams
// share the admitted, not-yet-running requests, each taking its part as one
// batch (a lone idle stream takes them all, up to the batch limits): one gather
// launch uploads their pinned host images (a copy-engine copy serves any other
// host buffer), one canny_run_batch runs them, one scatter launch writes the
// edge maps back. Several streams keep batches in flight at once, so new
// arrivals start while earlier ones are still on the GPU. A request completes
// when its batch's event fires; its latency is completion minus arrival, and
// its memory returns to the arena. The serial mode runs the same trace one
// request at a time through canny_run_pitched, as the baseline.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <thread>
#include <vector>

#include "canny_internal.cuh"
#include "serve_policy.h"

namespace canny {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device allocation; 256-byte granules.
class Arena {
public:
    bool init(size_t bytes)
    {
        bytes_ = bytes / 256 * 256;
        if (dev_alloc((void **)&base_, bytes_) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        free_[0] = bytes_;
        return true;
    }
    ~Arena()
    {
        if (base_) cudaFree(base_);
    }
    uint8_t *alloc(size_t n)
    {
        if (arena_failure_injected()) return nullptr;
        n = (n + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                used_ += n;
                peak_ = std::max(peak_, used_);
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(uint8_t *p, size_t n)
    {
        n = (n + 255) / 256 * 256;
        size_t off = (size_t)(p - base_);
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            free_.erase(next);
        }
        auto prev = free_.lower_bound(off);
        if (prev != free_.begin()) {
            --prev;
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t peak() const { return peak_; }

private:
    uint8_t *base_ = nullptr;
    size_t bytes_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Admitted {
    int req;
    uint8_t *in, *out;
    int pitch;
    size_t bytes;     // per buffer
};

struct Lane {
    cudaStream_t stream = nullptr;
    canny_ctx *ctx = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Admitted> running;
    // copy descriptors of the running batch: pinned staging and their device copies
    HostCopy *h_copies = nullptr, *d_copies = nullptr;   // [2 * cap]: inputs, then outputs
};

// Uploads (or downloads) the batch's images: one gather (scatter) launch for the
// pinned, tight, aligned host buffers, a copy-engine copy for any other.
cudaError_t move_images(Lane &L, const canny_request *reqs, int cap, bool upload)
{
    HostCopy *hc = L.h_copies + (upload ? 0 : cap);
    HostCopy *dc = L.d_copies + (upload ? 0 : cap);
    int n = 0;
    uint64_t words = 0;
    for (const Admitted &a : L.running) {
        const canny_request &r = reqs[a.req];
        uint8_t *host = upload ? const_cast<uint8_t *>(r.h_in) : r.h_out;
        const int hp = upload ? r.h_pitch : r.out_pitch;
        if (!host) continue;
        if (host_copy_ok(host, hp, r.w)) {
            hc[n++] = HostCopy{host, upload ? a.in : a.out, r.w, r.h, a.pitch, 0};
            words += host_copy_words(r.w, r.h);
            continue;
        }
        const cudaError_t e =
            upload ? cudaMemcpy2DAsync(a.in, a.pitch, host, hp, r.w, r.h, cudaMemcpyHostToDevice, L.stream)
                   : cudaMemcpy2DAsync(host, hp, a.out, a.pitch, r.w, r.h, cudaMemcpyDeviceToHost, L.stream);
        if (e != cudaSuccess) return e;
    }
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dc, hc, sizeof(HostCopy) * n, cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) return e;
    return upload ? launch_gather(dc, n, words, L.stream) : launch_scatter(dc, n, words, L.stream);
}

double pct(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

}  // namespace
}  // namespace canny

using namespace canny;

extern "C" canny_status canny_serve(const canny_serve_config *cfg, int n, const canny_request *reqs,
                                    double *latency_ms, canny_serve_report *out)
{
    if (!cfg || n < 0 || (n > 0 && !reqs) || !out) return CANNY_EINVAL;
    if (cfg->streams < 1 || cfg->max_batch_images < 1 || cfg->max_batch_images > 65535 || cfg->max_batch_pixels < 1 ||
        cfg->memory_budget_bytes <= 0)
        return CANNY_EINVAL;
    int64_t max_px = 0;
    int max_w = 1, max_h = 1;
    for (int i = 0; i < n; ++i) {
        const canny_request &r = reqs[i];
        if (r.w <= 0 || r.h <= 0 || !r.h_in || r.h_pitch < r.w || (r.h_out && r.out_pitch < r.w)) return CANNY_EINVAL;
        if (i > 0 && r.arrival_s < reqs[i - 1].arrival_s) return CANNY_EINVAL;   // arrival order
        // input + output buffers (16-byte pitched, 256-byte granules) must fit the budget
        const double need = 2.0 * (double)(((size_t)(r.w + 15) / 16 * 16 * (size_t)r.h + 255) / 256 * 256);
        if (need > cfg->memory_budget_bytes) return CANNY_EINVAL;
        max_px = std::max<int64_t>(max_px, (int64_t)r.w * r.h);
        max_w = std::max(max_w, r.w);
        max_h = std::max(max_h, r.h);
    }
    if (max_px > cfg->max_batch_pixels) return CANNY_EINVAL;
    *out = canny_serve_report{};
    if (n == 0) return CANNY_OK;

    canny_params p;
    canny_params_default(&p);
    p.low = (float)cfg->low;
    p.high = (float)cfg->high;
    Arena arena;
    if (!arena.init((size_t)cfg->memory_budget_bytes)) return CANNY_ENOMEM;

    // most tiles one batch can hold: its pixels in whole tiles plus a partial
    // row and column of tiles per image, and never more than the whole trace
    uint64_t trace_tiles = 0;
    for (int i = 0; i < n; ++i)
        trace_tiles += (uint64_t)((reqs[i].w + HT - 1) / HT) * (uint64_t)((reqs[i].h + HT - 1) / HT);
    const uint64_t per_image = (uint64_t)(max_w + HT - 1) / HT + (uint64_t)(max_h + HT - 1) / HT + 1;
    const uint64_t batch_bound = (uint64_t)cfg->max_batch_pixels / (HT * HT) +
                                 (uint64_t)std::min(cfg->max_batch_images, n) * per_image;
    const uint32_t batch_tiles = (uint32_t)std::min<uint64_t>({trace_tiles, batch_bound, 0x7fffffffull});
    const int nlanes = cfg->serial ? 1 : cfg->streams;
    std::vector<Lane> lanes(nlanes);
    canny_status st = CANNY_OK;
    for (auto &L : lanes) {
        if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
            st = CANNY_ECUDA;
            break;
        }
        // serial: one image at a time; batched: a pixel budget per batch
        const int64_t cap = cfg->serial ? max_px : cfg->max_batch_pixels;
        st = cfg->serial ? canny_create(max_w, max_h, &p, &L.ctx)
                         : canny_create((int)std::min<int64_t>(cap, 1 << 30), 1, &p, &L.ctx);
        if (st != CANNY_OK) break;
        const size_t cbytes = sizeof(HostCopy) * 2 * (size_t)cfg->max_batch_images;
        if (pinned_alloc((void **)&L.h_copies, cbytes) != cudaSuccess ||
            dev_alloc((void **)&L.d_copies, cbytes) != cudaSuccess) {
            cudaGetLastError();
            st = CANNY_ENOMEM;
            break;
        }
        if (cfg->band) {
            canny_tuning t = {cfg->band, cfg->ctas_per_sm, 0.0, 0, 0, 0, 0};
            st = canny_set_tuning(L.ctx, &t);
            if (st != CANNY_OK) break;
        }
        // size the lane for its largest possible batch now, so that no batch
        // grows the descriptor blob or the hysteresis scratch (each growth
        // synchronises the whole device, stalling every lane) while requests wait
        if (!cfg->serial) {
            st = batch_reserve(L.ctx, (uint32_t)std::min(cfg->max_batch_images, n), batch_tiles);
            if (st != CANNY_OK) break;
        }
    }

    std::vector<double> lat((size_t)n, 0.0);
    std::deque<int> waiting;                 // arrived, not yet admitted
    std::vector<Admitted> admitted;          // admitted, not yet running
    int next = 0, done = 0;
    int64_t batches = 0, batched_images = 0, deferrals = 0;
    const auto t0 = Clock::now();
    auto now_s = [&]() { return std::chrono::duration<double>(Clock::now() - t0).count(); };
    double last_done = 0.0;

    while (st == CANNY_OK && done < n) {
        const double now = now_s();
        while (next < n && reqs[next].arrival_s <= now) waiting.push_back(next++);
        // completions
        for (auto &L : lanes) {
            if (L.running.empty()) continue;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) { st = CANNY_ECUDA; break; }
            const double t = now_s();
            for (const Admitted &a : L.running) {
                lat[a.req] = (t - reqs[a.req].arrival_s) * 1e3;
                arena.release(a.in, a.bytes);
                arena.release(a.out, a.bytes);
            }
            done += (int)L.running.size();
            last_done = t;
            L.running.clear();
        }
        if (st != CANNY_OK) break;
        // admission in arrival order, as far as the memory budget allows
        while (!waiting.empty()) {
            const canny_request &r = reqs[waiting.front()];
            const int pitch = (r.w + 15) / 16 * 16;
            const size_t bytes = (size_t)pitch * (size_t)r.h;
            uint8_t *in = arena.alloc(bytes);
            if (!in) { ++deferrals; break; }
            uint8_t *o = arena.alloc(bytes);
            if (!o) { arena.release(in, bytes); ++deferrals; break; }
            admitted.push_back({waiting.front(), in, o, pitch, bytes});
            waiting.pop_front();
        }
        // the idle streams share the admitted requests (serve_policy.h)
        bool launched = false;
        int idle = 0;
        int64_t admitted_px = 0;
        for (const Lane &L : lanes) idle += L.running.empty() ? 1 : 0;
        auto px_of = [&](size_t i) { return (int64_t)reqs[admitted[i].req].w * reqs[admitted[i].req].h; };
        if (idle > 0)
            for (size_t i = 0; i < admitted.size(); ++i) admitted_px += px_of(i);
        for (auto &L : lanes) {
            if (!L.running.empty() || admitted.empty()) continue;
            std::vector<canny_image> imgs;
            const size_t k = batch_take(px_of, admitted.size(), cfg->max_batch_images, cfg->max_batch_pixels,
                                        batch_share(admitted_px, idle), cfg->serial != 0);
            for (size_t i = 0; i < k; ++i) admitted_px -= px_of(i);
            --idle;
            L.running.assign(admitted.begin(), admitted.begin() + (long)k);
            admitted.erase(admitted.begin(), admitted.begin() + (long)k);
            for (const Admitted &a : L.running) {
                const canny_request &r = reqs[a.req];
                imgs.push_back(canny_image{a.in, a.out, r.w, r.h, a.pitch, a.pitch});
            }
            if (move_images(L, reqs, cfg->max_batch_images, true) != cudaSuccess) { st = CANNY_ECUDA; break; }
            st = cfg->serial ? canny_run_pitched(L.ctx, &imgs[0], L.stream)
                             : canny_run_batch(L.ctx, (int)imgs.size(), imgs.data(), L.stream);
            if (st != CANNY_OK) break;
            if (move_images(L, reqs, cfg->max_batch_images, false) != cudaSuccess) st = CANNY_ECUDA;
            if (st == CANNY_OK && cudaEventRecord(L.done, L.stream) != cudaSuccess) st = CANNY_ECUDA;
            ++batches;
            batched_images += (int64_t)L.running.size();
            launched = true;
        }
        if (st != CANNY_OK) break;
        if (!launched) {
            // nothing to start: wait for the next arrival or a completion
            bool busy = false;
            for (auto &L : lanes) busy |= !L.running.empty();
            if (!busy && admitted.empty() && waiting.empty() && next < n) {
                const double dt = reqs[next].arrival_s - now_s();
                if (dt > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(dt - 1e-4));
            } else {
                std::this_thread::yield();
            }
        }
    }

    for (auto &L : lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        for (const Admitted &a : L.running) {
            arena.release(a.in, a.bytes);
            arena.release(a.out, a.bytes);
        }
        if (L.ctx) canny_destroy(L.ctx);
        if (L.h_copies) cudaFreeHost(L.h_copies);
        if (L.d_copies) cudaFree(L.d_copies);
        if (L.done) cudaEventDestroy(L.done);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    if (st != CANNY_OK) return st;

    int64_t px = 0;
    for (int i = 0; i < n; ++i) px += (int64_t)reqs[i].w * reqs[i].h;
    const double span = last_done - reqs[0].arrival_s;
    out->completed = done;
    out->wall_s = span;
    out->delivered_mpx_s = span > 0 ? (double)px / span / 1e6 : 0.0;
    out->p50_ms = pct(lat, 0.50);
    out->p99_ms = pct(lat, 0.99);
    out->max_ms = *std::max_element(lat.begin(), lat.end());
    out->batches = batches;
    out->mean_batch_images = batches ? (double)batched_images / (double)batches : 0.0;
    out->peak_bytes = (int64_t)arena.peak();
    out->deferrals = deferrals;
    if (latency_ms) std::copy(lat.begin(), lat.end(), latency_ms);
    return CANNY_OK;
}
