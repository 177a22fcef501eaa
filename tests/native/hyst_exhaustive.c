/*
 * Exhaustive check of the oracle's hysteresis (Step 4 of the paper's Sec. 2.2.1)
 * on every class map of a small shape, against an independent brute force:
 * start from the STRONG pixels and repeatedly add any WEAK pixel that has an
 * edge among its 8 neighbours, until nothing changes.
 *
 * usage: hyst_exhaustive W H   -> prints "checked N maps, M mismatches"
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void oracle_hysteresis(const uint8_t *cls, int w, int h, uint8_t *out, int out_pitch);

static void brute(const uint8_t *cls, int w, int h, uint8_t *edge)
{
    for (int i = 0; i < w * h; ++i) edge[i] = cls[i] == 2;
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                if (edge[y * w + x] || cls[y * w + x] != 1) continue;
                int hit = 0;
                for (int yy = y - 1; yy <= y + 1; ++yy)
                    for (int xx = x - 1; xx <= x + 1; ++xx)
                        if (yy >= 0 && yy < h && xx >= 0 && xx < w && edge[yy * w + xx]) hit = 1;
                if (hit) { edge[y * w + x] = 1; changed = 1; }
            }
    }
}

int main(int argc, char **argv)
{
    if (argc != 3) return 2;
    int w = atoi(argv[1]), h = atoi(argv[2]), n = w * h;
    if (n <= 0 || n > 20) return 2;
    uint8_t cls[20], out[20], edge[20];
    long long total = 1, bad = 0;
    for (int i = 0; i < n; ++i) total *= 3;
    for (long long code = 0; code < total; ++code) {
        long long c = code;
        for (int i = 0; i < n; ++i) { cls[i] = (uint8_t)(c % 3); c /= 3; }
        oracle_hysteresis(cls, w, h, out, w);
        brute(cls, w, h, edge);
        for (int i = 0; i < n; ++i)
            if ((out[i] == 255) != (edge[i] == 1) || (out[i] != 0 && out[i] != 255)) { ++bad; break; }
    }
    printf("checked %lld maps, %lld mismatches\n", total, bad);
    return bad != 0;
}
