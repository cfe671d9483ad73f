// Oracle: plain, single-threaded CPU definition of the k-mer counting result.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg may load this file's library.  It shares no
// code with the GPU library: it reads ASCII reads (never the 2-bit packed
// format), encodes each window from its characters, and keeps counts in a
// std::unordered_map.
//
// What it computes (the exact result the GPU path must reproduce bit for bit):
//
//  1. k-mers of a read of length M are its M-k+1 substrings of length k
//     (Section II-A).  A window that contains any character other than
//     A/C/G/T is skipped: the reads' quality screen (Section III-A) is read
//     as "drop windows over unknown bases".
//  2. Each base takes 2 bits, A=0 C=1 G=2 T=3, first base most significant, so
//     a k-mer is one 64-bit word (Section II-A: two bits per base, one 64-bit
//     number per k-mer) and numeric order equals lexicographic order.
//  3. A k-mer and its reverse complement are the same key: key = min(fwd, rc),
//     rc being the encoding of the reversed, complemented string.  (The paper
//     does not discuss strands; canonical keys are this library's reading.)
//  4. count[key][sample] = number of valid windows with that key, per sample.
//  5. The result keeps the keys whose count summed over samples is at least
//     min_count: k-mers that occur once are dropped (Section II-B, Count unit;
//     Section III, Prune), and Bloom false positives are removed (Section III,
//     Unify).  Keys are listed in ascending order.
//  6. The Bloom filter is the OR over every valid window of the window key's
//     bit pattern placed in one 64-bit word (a word-blocked filter):
//        h = mixer64(key), g = mixer64(h)
//        word   = h >> (64 - log2(bloom_bits / 64))
//        bit i  = (g >> 6i) & 63 for i < n_hashes   (colliding bits merge)
//     mixer64 is the SplitMix64 output function (Steele, Lea & Flood,
//     "Fast splittable pseudorandom number generators", OOPSLA 2014): add the
//     golden-ratio increment, then two xor-shift/multiply rounds and a final
//     xor-shift.  The paper names no hash function; this is the library's.
//
// Downstream of the count (Section II-B: the Count unit's table is read by
// the Filter unit; Section III-D: the table's 16-byte k-mer items):
//
//  7. 16-byte items: per result key, in ascending order, 8 bytes of key, then
//     the two per-sample counts as 16-bit numbers (both counts share 4 bytes
//     in the paper's item), each clamped to 65535, then 4 zero bytes of padding.
//     A one-sample job writes 0 as the second count.
//  8. Joint spectrum: hist[min(c0, cap) * (cap + 1) + min(c1, cap)] = number
//     of result keys with those clamped counts (two samples), hist[min(c0,
//     cap)] for one sample.
//  9. Filter selection (Section II-B, Filter unit: k-mers whose frequencies
//     differ between the samples).  The paper states no threshold; the
//     library's reading: with t the tumoral sample and n the other, a result
//     key is selected iff
//        count[t] >= min_tumor  and  count[n] <= max_normal  and
//        count[t] >= ratio * count[n]      (ratio 0: no ratio test).
// 10. Filter read hits (the Filter unit reads the input again and looks its
//     k-mers up in the table): hits[r] = number of valid windows of read r
//     whose key is selected; a read is a candidate iff hits[r] > 0.
// 11. Stem-grouped items (Section II-A: a k-mer's stem is its middle k-2
//     bases; Section III-D: the Filter unit's 72-byte item, 8 bytes of stem
//     and a 16-bit count per sample for each of the 16 k-mers that extend
//     the stem by one base on each side).  With canonical keys the library
//     reads it as: one item per canonical stem c (the smaller of a stem and
//     its reverse complement) that has a non-zero entry, ascending by c;
//     entry (x, y), stored at index 4*code(x) + code(y), holds the counts,
//     clamped to 65535, of the canonical key of the k-mer x c y (0 if that key
//     is not in the result).  Layout: 8 bytes of stem code, then 16 counts of
//     sample 0, then 16 of sample 1 (zero for one sample).  Needs k >= 3.
// 12. Two-filter Prune chain (Section III, Prune unit: every k-mer goes into
//     a first filter; one already present there, or a false positive, goes
//     into a second filter, which then holds the k-mers seen more than once;
//     the Count unit counts only k-mers found in the second filter).  The
//     second filter's content depends on the order of the insertions: a key
//     seen once lands in it only if other keys set all its bits in the first
//     filter before it.  For every order of the windows it lies between
//        lower = OR of pattern(key) at word(key) over keys with summed count >= 2
//        upper = lower OR, for every key with summed count 1 whose pattern is
//                inside the OR of the other keys' patterns at its word, its
//                pattern at its word
//     (same words and patterns as item 6).  The counting result is the same
//     as without the chain: the count pass is exact for the keys of the
//     second filter and keeps those whose count reaches min_count.
//
// Partition-restricted runs (for inputs too large to count in full here):
// when a keep-set over the top q bits of h is given, windows whose key falls
// outside the set are counted in the window total but not otherwise.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

int base_code(char c) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: return -1;
    }
}

char complement_base(char c) {
    switch (c) {
        case 'A': return 'T';
        case 'C': return 'G';
        case 'G': return 'C';
        case 'T': return 'A';
        default: return 'N';
    }
}

uint64_t mixer64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Encode k characters starting at s, first character most significant.
uint64_t encode(const char* s, int k) {
    uint64_t v = 0;
    for (int t = 0; t < k; ++t) v = v * 4 + (uint64_t)base_code(s[t]);
    return v;
}

int log2_exact(uint64_t x) {
    int r = 0;
    while ((1ull << r) < x) ++r;
    return r;
}

struct Oracle {
    int k;
    int n_samples;
    uint64_t bloom_bits;
    int n_hashes;
    uint32_t min_count;
    int log2_words;

    int restrict_bits = 0;           // 0 = count every key
    std::vector<uint8_t> keep;       // 2^restrict_bits flags

    uint64_t windows = 0;            // valid windows seen, all samples
    uint64_t counted = 0;            // windows whose key was counted
    std::unordered_map<uint64_t, std::vector<uint32_t>> counts;
    std::vector<uint64_t> bloom;                    // full filter (unrestricted)
    std::unordered_map<uint64_t, uint64_t> bloom_words;  // touched words (restricted)

    uint64_t word_of(uint64_t key) const {
        uint64_t h = mixer64(key);
        return log2_words == 0 ? 0 : h >> (64 - log2_words);
    }

    uint64_t pattern_of(uint64_t key) const {
        uint64_t g = mixer64(mixer64(key));
        uint64_t p = 0;
        for (int i = 0; i < n_hashes; ++i) {
            int bit = (int)((g >> (6 * i)) & 63);
            p |= 1ull << bit;
        }
        return p;
    }

    bool kept(uint64_t key) const {
        if (restrict_bits == 0) return true;
        return keep[mixer64(key) >> (64 - restrict_bits)] != 0;
    }

    void bloom_insert(uint64_t key) {
        uint64_t w = word_of(key);
        uint64_t g = mixer64(mixer64(key));
        for (int i = 0; i < n_hashes; ++i) {
            int bit = (int)((g >> (6 * i)) & 63);
            if (restrict_bits == 0)
                bloom[w] |= 1ull << bit;
            else
                bloom_words[w] |= 1ull << bit;
        }
    }

    void add_read(int sample, const char* s, uint64_t len) {
        if (len < (uint64_t)k) return;
        std::vector<char> rc_buf((size_t)k);
        for (uint64_t j = 0; j + (uint64_t)k <= len; ++j) {
            bool valid = true;
            for (int t = 0; t < k; ++t)
                if (base_code(s[j + t]) < 0) {
                    valid = false;
                    break;
                }
            if (!valid) continue;
            ++windows;
            uint64_t fwd = encode(s + j, k);
            for (int t = 0; t < k; ++t) rc_buf[t] = complement_base(s[j + k - 1 - t]);
            uint64_t rc = encode(rc_buf.data(), k);
            uint64_t key = std::min(fwd, rc);
            if (!kept(key)) continue;
            ++counted;
            auto& c = counts[key];
            if (c.empty()) c.assign((size_t)n_samples, 0u);
            if (c[sample] != 0xffffffffu) ++c[sample];
            bloom_insert(key);
        }
    }

    bool selected(const std::vector<uint32_t>& c, int tumor, uint32_t min_tumor, uint32_t max_normal,
                  uint32_t ratio) const {
        uint64_t t = c[tumor], n = c[1 - tumor];
        if (t < min_tumor) return false;
        if (n > max_normal) return false;
        if (t < (uint64_t)ratio * n) return false;
        return true;
    }

    // Result keys selected by the filter, ascending.
    std::vector<uint64_t> filter_keys(int tumor, uint32_t min_tumor, uint32_t max_normal, uint32_t ratio) const {
        std::vector<uint64_t> out;
        for (uint64_t key : result_keys())
            if (selected(counts.at(key), tumor, min_tumor, max_normal, ratio)) out.push_back(key);
        return out;
    }

    std::vector<uint64_t> result_keys() const {
        std::vector<uint64_t> keys;
        for (const auto& kv : counts) {
            uint64_t total = 0;
            for (uint32_t c : kv.second) total += c;
            if (total >= min_count) keys.push_back(kv.first);
        }
        std::sort(keys.begin(), keys.end());
        return keys;
    }
};

}  // namespace

extern "C" {

// Returns nullptr on invalid arguments (same ranges as the GPU library).
void* orc_create(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count) {
    if (k < 1 || k > 31 || n_samples < 1 || n_samples > 2 || n_hashes < 1 || n_hashes > 10 || min_count < 1)
        return nullptr;
    if (bloom_bits < 4096 || (bloom_bits & (bloom_bits - 1)) != 0) return nullptr;
    Oracle* o = new Oracle();
    o->k = k;
    o->n_samples = n_samples;
    o->bloom_bits = bloom_bits;
    o->n_hashes = n_hashes;
    o->min_count = min_count;
    o->log2_words = log2_exact(bloom_bits / 64);
    return o;
}

// Restrict counting to keys whose top q bits of mixer64(key) are flagged in
// keep[0 .. 2^q).  Must be called before the first orc_add_reads.
int orc_restrict(void* h, int q, const uint8_t* keep) {
    Oracle* o = (Oracle*)h;
    if (!o || q < 1 || q > 24 || !keep || o->windows != 0) return -1;
    o->restrict_bits = q;
    o->keep.assign(keep, keep + (1ull << q));
    return 0;
}

// Add n_reads ASCII reads of one sample; read r = ascii[offsets[r] .. offsets[r+1]).
int orc_add_reads(void* h, int sample, const char* ascii, const uint64_t* offsets, uint64_t n_reads) {
    Oracle* o = (Oracle*)h;
    if (!o || sample < 0 || sample >= o->n_samples || !offsets) return -1;
    if (!ascii && n_reads && offsets[n_reads] != offsets[0]) return -1;
    if (o->restrict_bits == 0 && o->bloom.empty()) o->bloom.assign(o->bloom_bits / 64, 0ull);
    for (uint64_t r = 0; r < n_reads; ++r) {
        if (offsets[r + 1] < offsets[r]) return -2;
        o->add_read(sample, ascii + offsets[r], offsets[r + 1] - offsets[r]);
    }
    return 0;
}

uint64_t orc_windows(void* h) { return ((Oracle*)h)->windows; }
uint64_t orc_counted(void* h) { return ((Oracle*)h)->counted; }
uint64_t orc_distinct(void* h) { return ((Oracle*)h)->counts.size(); }

// Number of keys in the result (count summed over samples >= min_count).
uint64_t orc_result_size(void* h) { return ((Oracle*)h)->result_keys().size(); }

// Write the result in ascending key order: keys[i], counts[i*n_samples + s].
int64_t orc_result(void* h, uint64_t* keys, uint32_t* counts, uint64_t capacity) {
    Oracle* o = (Oracle*)h;
    std::vector<uint64_t> ks = o->result_keys();
    if (ks.size() > capacity) return -1;
    for (size_t i = 0; i < ks.size(); ++i) {
        keys[i] = ks[i];
        const auto& c = o->counts.at(ks[i]);
        for (int s = 0; s < o->n_samples; ++s) counts[i * o->n_samples + s] = c[s];
    }
    return (int64_t)ks.size();
}

// Copy Bloom words [first, first + n) (words never set read as 0).
int orc_bloom(void* h, uint64_t* out, uint64_t first, uint64_t n) {
    Oracle* o = (Oracle*)h;
    uint64_t nw = o->bloom_bits / 64;
    if (first > nw || n > nw - first) return -1;
    for (uint64_t i = 0; i < n; ++i) {
        if (o->restrict_bits == 0) {
            out[i] = o->bloom.empty() ? 0 : o->bloom[first + i];
        } else {
            auto it = o->bloom_words.find(first + i);
            out[i] = it == o->bloom_words.end() ? 0 : it->second;
        }
    }
    return 0;
}

// 1 if every bit of key's pattern is set in its word (membership query).
int orc_bloom_query(void* h, uint64_t key) {
    Oracle* o = (Oracle*)h;
    uint64_t w = o->word_of(key), p = o->pattern_of(key);
    uint64_t word = 0;
    if (o->restrict_bits == 0) {
        word = o->bloom.empty() ? 0 : o->bloom[w];
    } else {
        auto it = o->bloom_words.find(w);
        word = it == o->bloom_words.end() ? 0 : it->second;
    }
    return (word & p) == p ? 1 : 0;
}

uint64_t orc_bloom_word_index(void* h, uint64_t key) { return ((Oracle*)h)->word_of(key); }
uint64_t orc_bloom_pattern(void* h, uint64_t key) { return ((Oracle*)h)->pattern_of(key); }
uint64_t orc_mixer64(uint64_t x) { return mixer64(x); }

// Partition (top q bits of mixer64) of each of n keys, for restricted comparisons.
int orc_partitions(const uint64_t* keys, uint64_t n, int q, uint32_t* out) {
    if (q < 1 || q > 24 || (!keys && n) || (!out && n)) return -1;
    for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)(mixer64(keys[i]) >> (64 - q));
    return 0;
}

// Canonical key of the k characters at s, or ~0 if any is not A/C/G/T.
uint64_t orc_canonical(const char* s, int k) {
    for (int t = 0; t < k; ++t)
        if (base_code(s[t]) < 0) return ~0ull;
    std::vector<char> rc((size_t)k);
    for (int t = 0; t < k; ++t) rc[t] = complement_base(s[k - 1 - t]);
    return std::min(encode(s, k), encode(rc.data(), k));
}

// 16-byte items of the result (item 7 above): 16 bytes per key written to out
// (little-endian fields at byte offsets 0, 8, 10, 12).  Returns the number of
// items, -1 if capacity (in items) is too small.
int64_t orc_items16(void* h, uint8_t* out, uint64_t capacity) {
    Oracle* o = (Oracle*)h;
    std::vector<uint64_t> ks = o->result_keys();
    if (ks.size() > capacity) return -1;
    for (size_t i = 0; i < ks.size(); ++i) {
        const auto& c = o->counts.at(ks[i]);
        uint16_t c16[2] = {0, 0};
        for (int s = 0; s < o->n_samples; ++s) c16[s] = c[s] > 65535u ? 65535u : (uint16_t)c[s];
        uint32_t pad = 0;
        uint8_t* item = out + 16 * i;
        std::memcpy(item, &ks[i], 8);
        std::memcpy(item + 8, &c16[0], 2);
        std::memcpy(item + 10, &c16[1], 2);
        std::memcpy(item + 12, &pad, 4);
    }
    return (int64_t)ks.size();
}

// Joint spectrum of the result (item 8): hist has (cap+1)^n_samples entries.
int orc_spectrum(void* h, uint32_t cap, uint64_t* hist) {
    Oracle* o = (Oracle*)h;
    if (!o || cap < 1 || !hist) return -1;
    const uint64_t side = (uint64_t)cap + 1;
    const uint64_t n_bins = o->n_samples == 2 ? side * side : side;
    for (uint64_t b = 0; b < n_bins; ++b) hist[b] = 0;
    for (uint64_t key : o->result_keys()) {
        const auto& c = o->counts.at(key);
        uint64_t bin = std::min<uint64_t>(c[0], cap);
        if (o->n_samples == 2) bin = bin * side + std::min<uint64_t>(c[1], cap);
        ++hist[bin];
    }
    return 0;
}

// Filter selection (item 9): keys and counts (n_samples per key) of the
// selected result keys, ascending.  keys == nullptr: size only.  Returns the
// number of keys; -1 for invalid arguments or too small a capacity.
int64_t orc_filter_select(void* h, int tumor, uint32_t min_tumor, uint32_t max_normal, uint32_t ratio,
                          uint64_t* keys, uint32_t* counts, uint64_t capacity) {
    Oracle* o = (Oracle*)h;
    if (!o || o->n_samples != 2 || tumor < 0 || tumor > 1) return -1;
    std::vector<uint64_t> ks = o->filter_keys(tumor, min_tumor, max_normal, ratio);
    if (!keys) return (int64_t)ks.size();
    if (ks.size() > capacity) return -1;
    for (size_t i = 0; i < ks.size(); ++i) {
        keys[i] = ks[i];
        const auto& c = o->counts.at(ks[i]);
        counts[2 * i] = c[0];
        counts[2 * i + 1] = c[1];
    }
    return (int64_t)ks.size();
}

// Filter read hits (item 10) of n_reads ASCII reads: hits[r] per read.
// Returns the number of candidate reads (hits > 0), -1 on invalid arguments.
int64_t orc_filter_reads(void* h, int tumor, uint32_t min_tumor, uint32_t max_normal, uint32_t ratio,
                         const char* ascii, const uint64_t* offsets, uint64_t n_reads, uint32_t* hits) {
    Oracle* o = (Oracle*)h;
    if (!o || o->n_samples != 2 || tumor < 0 || tumor > 1 || !offsets || (n_reads && !hits)) return -1;
    if (!ascii && n_reads && offsets[n_reads] != offsets[0]) return -1;
    std::vector<uint64_t> ks = o->filter_keys(tumor, min_tumor, max_normal, ratio);
    std::unordered_map<uint64_t, bool> sel;
    for (uint64_t key : ks) sel[key] = true;
    const int k = o->k;
    std::vector<char> rc_buf((size_t)k);
    int64_t candidates = 0;
    for (uint64_t r = 0; r < n_reads; ++r) {
        if (offsets[r + 1] < offsets[r]) return -1;
        const char* s = ascii + offsets[r];
        const uint64_t len = offsets[r + 1] - offsets[r];
        uint32_t n_hits = 0;
        for (uint64_t j = 0; len >= (uint64_t)k && j + (uint64_t)k <= len; ++j) {
            bool valid = true;
            for (int t = 0; t < k; ++t)
                if (base_code(s[j + t]) < 0) {
                    valid = false;
                    break;
                }
            if (!valid) continue;
            for (int t = 0; t < k; ++t) rc_buf[t] = complement_base(s[j + k - 1 - t]);
            const uint64_t key = std::min(encode(s + j, k), encode(rc_buf.data(), k));
            if (sel.count(key)) ++n_hits;
        }
        hits[r] = n_hits;
        if (n_hits) ++candidates;
    }
    return candidates;
}

// Stem-grouped items (item 11): 72 bytes per item into out.  Every result
// key is spelled out as a string in both orientations; an orientation whose
// stem is canonical (not larger than its reverse complement) fills entry
// (first base, last base) of that stem's item.  Returns the number of items,
// -1 if k < 3 or capacity (in items) is too small; out == nullptr: size only.
int64_t orc_stems(void* h, uint8_t* out, uint64_t capacity) {
    Oracle* o = (Oracle*)h;
    if (!o || o->k < 3) return -1;
    const int k = o->k;
    const char letters[4] = {'A', 'C', 'G', 'T'};
    struct Item {
        uint16_t c[2][16];
    };
    std::map<uint64_t, Item> items;
    for (uint64_t key : o->result_keys()) {
        std::string fwd((size_t)k, 'A');
        for (int t = 0; t < k; ++t) fwd[t] = letters[(key >> (2 * (k - 1 - t))) & 3];
        std::string rc((size_t)k, 'A');
        for (int t = 0; t < k; ++t) rc[t] = complement_base(fwd[k - 1 - t]);
        const auto& cnt = o->counts.at(key);
        for (const std::string& kmer : {fwd, rc}) {
            const std::string stem = kmer.substr(1, k - 2);
            std::string stem_rc(stem.size(), 'A');
            for (size_t t = 0; t < stem.size(); ++t) stem_rc[t] = complement_base(stem[stem.size() - 1 - t]);
            if (stem > stem_rc) continue;  // not the canonical stem: the other orientation fills the entry
            const uint64_t code = encode(stem.data(), k - 2);
            Item& it = items[code];  // value-initialised: all counts 0
            const int e = 4 * base_code(kmer[0]) + base_code(kmer[k - 1]);
            for (int s = 0; s < o->n_samples; ++s) it.c[s][e] = cnt[s] > 65535u ? 65535u : (uint16_t)cnt[s];
        }
    }
    if (!out) return (int64_t)items.size();
    if (items.size() > capacity) return -1;
    size_t i = 0;
    for (const auto& kv : items) {
        uint8_t* item = out + 72 * i++;
        std::memcpy(item, &kv.first, 8);
        std::memcpy(item + 8, kv.second.c, 64);
    }
    return (int64_t)items.size();
}

// Bounds of the Prune chain's second filter (item 12), words [first, first +
// n) of each.  Unrestricted runs only.  Returns 0, or -1 for a bad range.
int orc_bloom2_bounds(void* h, uint64_t* lower, uint64_t* upper, uint64_t first, uint64_t n) {
    Oracle* o = (Oracle*)h;
    const uint64_t nw = o->bloom_bits / 64;
    if (o->restrict_bits != 0 || first > nw || n > nw - first) return -1;
    std::unordered_map<uint64_t, std::vector<uint64_t>> by_word;  // word -> keys counted there
    for (const auto& kv : o->counts) by_word[o->word_of(kv.first)].push_back(kv.first);
    for (uint64_t i = 0; i < n; ++i) lower[i] = upper[i] = 0;
    for (const auto& wk : by_word) {
        const uint64_t w = wk.first;
        if (w < first || w >= first + n) continue;
        uint64_t lo = 0, hi = 0;
        for (uint64_t key : wk.second) {
            uint64_t total = 0;
            for (uint32_t c : o->counts.at(key)) total += c;
            const uint64_t pat = o->pattern_of(key);
            if (total >= 2) {
                lo |= pat;
                hi |= pat;
                continue;
            }
            uint64_t others = 0;
            for (uint64_t other : wk.second)
                if (other != key) others |= o->pattern_of(other);
            if ((others & pat) == pat) hi |= pat;
        }
        lower[w - first] = lo;
        upper[w - first] = hi;
    }
    return 0;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

}  // extern "C"
