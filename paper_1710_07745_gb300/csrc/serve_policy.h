// serve_policy.h -- which admitted requests an idle stream of canny_serve takes
// as its batch (plain C++, no CUDA: the serving loop and its host tests share it).
//
// The admitted, not-yet-running requests wait in arrival order. When several
// streams are idle they share them: each idle stream in turn takes a prefix
// worth about an equal part of the waiting pixels, so that requests arriving
// together run side by side instead of all waiting for the largest image of
// one batch. A stream that is the only idle one takes everything the batch
// limits allow.
#pragma once

#include <cstddef>
#include <cstdint>

namespace canny {

// The pixels an idle stream aims for when `idle` streams share `waiting_px`
// pixels of admitted requests (rounded up, so the shares cover every pixel).
inline int64_t batch_share(int64_t waiting_px, int idle)
{
    return idle > 1 ? (waiting_px + idle - 1) / idle : waiting_px;
}

// How many of the n admitted requests (pixels px(0), px(1), ... in arrival
// order) one idle stream takes: the longest prefix within max_images requests
// and max_pixels pixels that goes past `share` pixels only with its first
// request; at least one request whenever n > 0 and the first one fits
// max_pixels. serial: one request at most.
template <class Px>
size_t batch_take(Px px, size_t n, int max_images, int64_t max_pixels, int64_t share, bool serial)
{
    size_t k = 0;
    int64_t sum = 0;
    for (; k < n; ++k) {
        const int64_t a = px(k);
        if ((int64_t)k >= (int64_t)max_images || sum + a > max_pixels || (serial && k >= 1)) break;
        if (k > 0 && sum + a > share) break;
        sum += a;
    }
    return k;
}

}  // namespace canny
