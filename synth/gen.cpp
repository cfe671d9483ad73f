// Seeded synthetic DNA workloads: genomes, mutated copies and sequencing reads.
//
// This module only draws random inputs.  It holds none of the counting
// method's arithmetic (no k-mer encoding, no hashing, no Bloom filter), so both
// the CPU oracle and the GPU library can be fed from it without sharing code.
//
// Random numbers come from xoshiro256** (Blackman & Vigna, "Scrambled linear
// pseudorandom number generators", 2018), written here from its published
// definition.  Every block of work owns a stream seeded from (seed, stream id,
// block index), so the output does not depend on the number of threads.
//
// Output format: ASCII bytes over {A,C,G,T,N}; reads are concatenated and
// described by offsets[n_reads + 1] (read r = bytes [offsets[r], offsets[r+1])).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct Xoshiro256ss {
    uint64_t s[4];

    static uint64_t rotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

    // State expansion: a 64-bit LCG (Knuth's MMIX constants) whose outputs are
    // scrambled by an xorshift; any seed gives a non-zero state.
    Xoshiro256ss(uint64_t seed, uint64_t stream, uint64_t block) {
        uint64_t x = seed * 0x100000001b3ull ^ (stream + 0x51ed270b27bd5e4full) * 0x2545f4914f6cdd1dull ^
                     (block + 1) * 0x9fb21c651e98df25ull;
        for (int i = 0; i < 4; ++i) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            uint64_t z = x;
            z ^= z >> 33;
            z *= 0xff51afd7ed558ccdull;
            z ^= z >> 29;
            s[i] = z | (i == 0 ? 1ull : 0ull);
        }
        for (int i = 0; i < 16; ++i) next();  // decorrelate nearby seeds
    }

    uint64_t next() {
        const uint64_t result = rotl(s[1] * 5, 7) * 9;
        const uint64_t t = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= t;
        s[3] = rotl(s[3], 45);
        return result;
    }

    // Uniform integer in [0, n) by multiply-shift (Lemire); bias < n / 2^64.
    uint64_t below(uint64_t n) { return (uint64_t)(((unsigned __int128)next() * n) >> 64); }
};

const char kBases[4] = {'A', 'C', 'G', 'T'};

char complement_ascii(char c) {
    switch (c) {
        case 'A': return 'T';
        case 'C': return 'G';
        case 'G': return 'C';
        case 'T': return 'A';
        default: return 'N';
    }
}

// Threshold for an event of probability p tested against a uniform 32-bit draw.
uint64_t threshold32(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return 1ull << 32;
    return (uint64_t)(p * 4294967296.0);
}

template <class F>
void parallel_blocks(uint64_t n_blocks, int threads, F&& f) {
    if (threads <= 1 || n_blocks <= 1) {
        for (uint64_t b = 0; b < n_blocks; ++b) f(b);
        return;
    }
    int nt = (int)std::min<uint64_t>((uint64_t)threads, n_blocks);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) {
        pool.emplace_back([&, t]() {
            for (uint64_t b = (uint64_t)t; b < n_blocks; b += (uint64_t)nt) f(b);
        });
    }
    for (auto& th : pool) th.join();
}

constexpr uint64_t kGenomeBlock = 1ull << 20;  // bases per genome stream block
constexpr uint64_t kReadBlock = 1ull << 14;    // reads per read stream block

enum : uint64_t { kStreamGenome = 1, kStreamLengths = 2, kStreamReads = 3, kStreamMutate = 4 };

}  // namespace

extern "C" {

// Fill out[0..G) with i.i.d. uniform bases A/C/G/T.
int synth_genome(uint64_t seed, uint64_t G, uint8_t* out, int threads) {
    if (!out && G) return -1;
    uint64_t n_blocks = (G + kGenomeBlock - 1) / kGenomeBlock;
    parallel_blocks(n_blocks, threads, [&](uint64_t b) {
        Xoshiro256ss rng(seed, kStreamGenome, b);
        uint64_t lo = b * kGenomeBlock, hi = std::min(G, lo + kGenomeBlock);
        uint64_t word = 0;
        int left = 0;
        for (uint64_t i = lo; i < hi; ++i) {
            if (left == 0) {
                word = rng.next();
                left = 32;
            }
            out[i] = (uint8_t)kBases[word & 3];
            word >>= 2;
            --left;
        }
    });
    return 0;
}

// Copy genome g into out while injecting single-base substitutions (rate
// snv_rate per base) and insertions/deletions (rate indel_rate per base,
// lengths uniform in [1, indel_max], insert or delete with equal odds).
// Returns the new length, or -1 when cap is too small.
int64_t synth_mutate(uint64_t seed, const uint8_t* g, uint64_t G, double snv_rate, double indel_rate,
                     int indel_max, uint8_t* out, uint64_t cap) {
    Xoshiro256ss rng(seed, kStreamMutate, 0);
    const uint64_t t_snv = threshold32(snv_rate), t_indel = threshold32(indel_rate);
    uint64_t o = 0;
    for (uint64_t i = 0; i < G; ++i) {
        uint64_t r = rng.next();
        char c = (char)g[i];
        if ((r & 0xffffffffull) < t_snv) {
            int code = c == 'A' ? 0 : c == 'C' ? 1 : c == 'G' ? 2 : 3;
            c = kBases[(code + 1 + (int)rng.below(3)) & 3];
        }
        if (o >= cap) return -1;
        out[o++] = (uint8_t)c;
        if ((r >> 32) < t_indel) {
            uint64_t len = 1 + rng.below((uint64_t)std::max(1, indel_max));
            if (rng.next() & 1) {
                for (uint64_t j = 0; j < len; ++j) {
                    if (o >= cap) return -1;
                    out[o++] = (uint8_t)kBases[rng.below(4)];
                }
            } else {
                i += len;  // skip the next len bases of the source
            }
        }
    }
    return (int64_t)o;
}

// offsets[0..n_reads] = running sum of read lengths, each uniform in
// [len_min, len_max] (offsets[0] = 0).
int synth_read_offsets(uint64_t seed, uint64_t n_reads, uint32_t len_min, uint32_t len_max, uint64_t* offsets,
                       int threads) {
    if (len_min > len_max || !offsets) return -1;
    uint64_t n_blocks = (n_reads + kReadBlock - 1) / kReadBlock;
    const uint64_t span = (uint64_t)(len_max - len_min) + 1;
    parallel_blocks(n_blocks, threads, [&](uint64_t b) {
        Xoshiro256ss rng(seed, kStreamLengths, b);
        uint64_t lo = b * kReadBlock, hi = std::min(n_reads, lo + kReadBlock);
        for (uint64_t r = lo; r < hi; ++r) offsets[r + 1] = len_min + (span > 1 ? rng.below(span) : 0);
    });
    offsets[0] = 0;
    for (uint64_t r = 0; r < n_reads; ++r) offsets[r + 1] += offsets[r];
    return 0;
}

// Sample reads from genome[0..G): read r has length offsets[r+1]-offsets[r],
// starts uniformly in [0, G - len], comes from either strand with equal odds
// (reverse complement for the minus strand), then each base is substituted
// with probability sub_rate (uniformly to one of the three other bases) and
// finally replaced by 'N' with probability n_rate.
int synth_reads(uint64_t seed, const uint8_t* genome, uint64_t G, uint64_t n_reads, double sub_rate,
                double n_rate, const uint64_t* offsets, uint8_t* out, int threads) {
    if (!genome || !offsets || !out) return -1;
    for (uint64_t r = 0; r < n_reads; ++r)
        if (offsets[r + 1] - offsets[r] > G) return -2;
    const uint64_t t_sub = threshold32(sub_rate), t_n = threshold32(n_rate);
    uint64_t n_blocks = (n_reads + kReadBlock - 1) / kReadBlock;
    parallel_blocks(n_blocks, threads, [&](uint64_t b) {
        Xoshiro256ss rng(seed, kStreamReads, b);
        uint64_t lo = b * kReadBlock, hi = std::min(n_reads, lo + kReadBlock);
        for (uint64_t r = lo; r < hi; ++r) {
            uint64_t len = offsets[r + 1] - offsets[r];
            uint8_t* dst = out + offsets[r];
            uint64_t start = rng.below(G - len + 1);
            bool minus = rng.next() & 1;
            for (uint64_t j = 0; j < len; ++j) {
                char c = minus ? complement_ascii((char)genome[start + len - 1 - j]) : (char)genome[start + j];
                uint64_t u = rng.next();
                if ((u & 0xffffffffull) < t_sub) {
                    int code = c == 'A' ? 0 : c == 'C' ? 1 : c == 'G' ? 2 : 3;
                    c = kBases[(code + 1 + (int)rng.below(3)) & 3];
                }
                if ((u >> 32) < t_n) c = 'N';
                dst[j] = (uint8_t)c;
            }
        }
    });
    return 0;
}

}  // extern "C"
