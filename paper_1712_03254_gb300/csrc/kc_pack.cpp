// Host helper: ASCII bases -> the packed read format of include/kc.h.
// Base i goes to bits [63-2(i%32) .. 62-2(i%32)] of packed[i/32] with
// A=0 C=1 G=2 T=3; any other byte sets bit 63-(i%64) of n_mask[i/64] and is
// stored with code 0.

#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

#include "../../include/kc.h"

namespace {

struct CodeTable {
    uint8_t code[256];
    uint8_t unknown[256];
    CodeTable() {
        for (int c = 0; c < 256; ++c) {
            code[c] = 0;
            unknown[c] = 1;
        }
        const char bases[4] = {'A', 'C', 'G', 'T'};
        for (int i = 0; i < 4; ++i) {
            code[(uint8_t)bases[i]] = (uint8_t)i;
            unknown[(uint8_t)bases[i]] = 0;
        }
    }
};

const CodeTable kTable;

void pack_range(const uint8_t* a, uint64_t n_bases, uint64_t w64_lo, uint64_t w64_hi, uint64_t* packed,
                uint64_t* n_mask) {
    for (uint64_t w = w64_lo; w < w64_hi; ++w) {
        uint64_t p0 = 0, p1 = 0, m = 0;
        const uint64_t base = w * 64;
        const uint64_t end = std::min<uint64_t>(64, n_bases - base);
        for (uint64_t t = 0; t < end; ++t) {
            const uint8_t c = a[base + t];
            const uint64_t code = kTable.code[c];
            if (t < 32)
                p0 |= code << (62 - 2 * t);
            else
                p1 |= code << (62 - 2 * (t - 32));
            m |= (uint64_t)kTable.unknown[c] << (63 - t);
        }
        packed[2 * w] = p0;
        if (end > 32) packed[2 * w + 1] = p1;
        n_mask[w] = m;
    }
}

}  // namespace

extern "C" kc_status kc_pack_ascii(const char* ascii, uint64_t n_bases, uint64_t* packed, uint64_t* n_mask) {
    if (n_bases == 0) return KC_OK;
    if (!ascii || !packed || !n_mask) return KC_ERR_ARG;
    const uint8_t* a = reinterpret_cast<const uint8_t*>(ascii);
    const uint64_t n_w64 = (n_bases + 63) / 64;
    const uint64_t per = 1ull << 14;  // 64-base words per task
    const uint64_t n_tasks = (n_w64 + per - 1) / per;
    unsigned hw = std::thread::hardware_concurrency();
    const uint64_t nt = std::min<uint64_t>(n_tasks, hw ? std::min(hw, 32u) : 1u);
    auto run = [&](uint64_t t0) {
        for (uint64_t t = t0; t < n_tasks; t += nt)
            pack_range(a, n_bases, t * per, std::min(n_w64, (t + 1) * per), packed, n_mask);
    };
    if (nt <= 1) {
        run(0);
    } else {
        std::vector<std::thread> pool;
        for (uint64_t t = 0; t < nt; ++t) pool.emplace_back(run, t);
        for (auto& th : pool) th.join();
    }
    return KC_OK;
}
