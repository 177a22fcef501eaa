// Property checks of the serving loop's batch policy (serve_policy.h), run on
// the host: random queues of admitted requests shared out to the idle streams
// the way canny_serve does it. Prints every violation; exits 1 if there was any.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "serve_policy.h"

namespace {

uint64_t rng_state = 0x9E3779B97F4A7C15ull;

uint64_t next_u64()   // splitmix64
{
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int64_t uniform(int64_t lo, int64_t hi) { return lo + (int64_t)(next_u64() % (uint64_t)(hi - lo + 1)); }

int failures = 0;

void fail(const char *what, int trial)
{
    if (failures < 20) std::printf("trial %d: %s\n", trial, what);
    ++failures;
}

}  // namespace

int main()
{
    using canny::batch_share;
    using canny::batch_take;

    // batch_share: the idle streams' shares cover the waiting pixels, none above them
    for (int trial = 0; trial < 10000; ++trial) {
        const int64_t w = uniform(0, 1ll << 40);
        const int idle = (int)uniform(1, 64);
        const int64_t s = batch_share(w, idle);
        if (s * idle < w) fail("shares do not cover the waiting pixels", trial);
        if (s > w) fail("a share exceeds the waiting pixels", trial);
    }

    for (int trial = 0; trial < 20000; ++trial) {
        const size_t n = (size_t)uniform(0, 300);
        const int64_t max_px = uniform(1, 1 << 22);
        std::vector<int64_t> px(n);
        for (auto &p : px) p = uniform(1, max_px);           // every request fits a batch alone
        const int max_images = (int)uniform(1, 400);
        const int64_t max_pixels = max_px + uniform(0, 1 << 24);
        const bool serial = uniform(0, 9) == 0;
        const int idle0 = (int)uniform(1, 8);

        size_t head = 0;
        int64_t waiting = 0;
        for (int64_t p : px) waiting += p;
        int idle = idle0;
        while (idle > 0 && head < n) {
            const int64_t share = batch_share(waiting, idle);
            auto at = [&](size_t i) { return px[head + i]; };
            const size_t k = batch_take(at, n - head, max_images, max_pixels, share, serial);
            int64_t sum = 0;
            for (size_t i = 0; i < k; ++i) sum += at(i);
            if (k < 1) fail("an idle stream took nothing from a non-empty queue", trial);
            if ((int64_t)k > max_images) fail("more images than the batch limit", trial);
            if (sum > max_pixels) fail("more pixels than the batch limit", trial);
            if (serial && k > 1) fail("serial mode took more than one request", trial);
            if (k > 1 && sum > share) fail("a batch of several requests went past its share", trial);
            if (head + k < n) {   // nothing more could have been taken
                const int64_t nx = at(k);
                const bool stop = (int64_t)k >= max_images || sum + nx > max_pixels || (serial && k >= 1) ||
                                  (k > 0 && sum + nx > share);
                if (!stop) fail("a batch stopped short of its limits and its share", trial);
            }
            // a lone idle stream takes what the batch limits allow (the policy
            // without sharing)
            if (idle == 1) {
                size_t lone = 0;
                int64_t s2 = 0;
                while (head + lone < n && (int64_t)lone < max_images && s2 + at(lone) <= max_pixels &&
                       !(serial && lone >= 1))
                    s2 += at(lone++);
                if (lone != k) fail("a lone idle stream did not take the whole batch", trial);
            }
            head += k;
            waiting -= sum;
            --idle;
        }
        // with limits that never bind, the idle streams take the whole queue
        int64_t total = 0;
        for (int64_t p : px) total += p;
        if (!serial && (int64_t)n <= max_images && total <= max_pixels && head != n)
            fail("requests left waiting beside idle streams", trial);
    }

    for (int trial = 0; trial < 2000; ++trial) {
        const int idle0 = (int)uniform(1, 8);
        const size_t per = (size_t)uniform(1, 40);
        const size_t n = per * (size_t)idle0;
        const int64_t size = uniform(1, 1 << 20);
        std::vector<int64_t> px(n, size);
        size_t head = 0;
        int64_t waiting = size * (int64_t)n;
        for (int idle = idle0; idle > 0; --idle) {
            auto at = [&](size_t i) { return px[head + i]; };
            const size_t k = batch_take(at, n - head, 1 << 20, 1ll << 50, batch_share(waiting, idle), false);
            if (k != per) fail("equal requests were not split evenly", trial);
            head += k;
            waiting -= (int64_t)k * size;
        }
        if (head != n) fail("equal requests left waiting", trial);
    }

    std::printf("%d failures\n", failures);
    return failures ? 1 : 0;
}
