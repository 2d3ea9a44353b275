// Host construction of the seeding front end's index (no CUDA: the library
// uploads the result, and a CPU test checks it against plain definitions).
//
// For a reference of L bases (2-bit packed, base p in bits 2*(p&15) of word
// p>>4) followed by a terminator smaller than every base, rows 0..L are the
// suffixes in order of their first 32 bases (a suffix with fewer bases before
// the terminator sorts before every longer one it prefixes; equal 32-base keys
// in position order).  That order is exact for every pattern of up to 32 bases.
//  - sa[row]: the suffix's position (row 0 is the empty suffix at L);
//  - occ: 16 words per chunk of 192 rows: the counts of A, C, G, T among the
//    BWT entries of the rows before the chunk, then the chunk's 192 two-bit BWT
//    entries as two bit planes of 6 words each (words 4..9 the low bits, 10..15
//    the high bits; bit k of word w is row 32w + k of the chunk), so the rows
//    holding one base are one mask per 32 rows (entry of row i = the base before
//    suffix sa[i]; the row of suffix 0 stores 0 and is not counted: its entry is
//    the terminator);
//  - C[c]: the first row of the suffixes that start with base c;
//  - lut[P]: the row interval [lo, hi) of the suffixes that start with the
//    12-base pattern P (first base most significant).
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <thread>
#include <vector>

namespace sa {

constexpr int kLutK = 12;                          // bases resolved by the lookup table
constexpr uint32_t kLutSize = 1u << (2 * kLutK);
constexpr int kChunkRows = 192;                    // BWT rows per 64-byte chunk
constexpr int kKeyBases = 32;                      // depth of the suffix order

struct RowInterval {
    uint32_t lo, hi;
};

struct __attribute__((packed)) SeedRec {
    uint64_t key;      // first 32 bases, 2 bits each, first base most significant, 0 past the end
    uint32_t tie;      // bases present (< 32: a suffix near the end, which sorts first among equal
                       // keys, shorter first); else 32 + position (equal keys in position order)
};

inline uint32_t seed_code_at(const uint32_t* w, uint64_t L, uint64_t q) {
    return q < L ? (w[q >> 4] >> (2 * (q & 15))) & 3u : 0u;
}
inline uint64_t seed_rec_pos(const SeedRec& r, uint64_t L) { return r.tie < kKeyBases ? L - r.tie : (uint64_t)r.tie - kKeyBases; }

template <class F>
inline void seed_parallel_ranges(uint64_t n, unsigned T, F&& fn) {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < T; t++) {
        const uint64_t a = n * t / T, b = n * (t + 1) / T;
        th.emplace_back([&, a, b, t] { fn(t, a, b); });
    }
    for (auto& x : th) x.join();
}

struct SeedHostIndex {
    std::vector<uint32_t> sa;
    std::vector<uint32_t> occ;     // 16 words per chunk
    std::vector<RowInterval> lut;
    uint32_t dollar_row = 0;
    uint32_t C[4] = {};
};

// Suffix order, BWT chunks and lookup table of the packed reference `w` (L bases).
inline void build_seed_index(const uint32_t* w, uint64_t L, SeedHostIndex& H) {
    const uint64_t rows = L + 1;
    const unsigned T = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    auto key_of = [&](uint64_t p) {
        uint64_t k = 0;
        for (int t = 0; t < kKeyBases; t++) k = (k << 2) | seed_code_at(w, L, p + t);
        return k;
    };
    auto tie_of = [&](uint64_t p) {
        return L - p < (uint64_t)kKeyBases ? (uint32_t)(L - p) : (uint32_t)(kKeyBases + p);
    };
    // 1. bucket by the first 8 bases (counting sort), then sort each bucket
    constexpr uint32_t NB = 1u << 16;
    std::vector<std::vector<uint64_t>> hist(T, std::vector<uint64_t>(NB, 0));
    seed_parallel_ranges(rows, T, [&](unsigned t, uint64_t a, uint64_t b) {
        if (a >= b) return;
        uint64_t k = key_of(a);
        for (uint64_t p = a; p < b; p++) {
            hist[t][k >> 48]++;
            k = (k << 2) | seed_code_at(w, L, p + kKeyBases);
        }
    });
    std::vector<uint64_t> bstart(NB + 1, 0);
    {
        uint64_t acc = 0;
        for (uint32_t bkt = 0; bkt < NB; bkt++) {
            bstart[bkt] = acc;
            for (unsigned t = 0; t < T; t++) {
                const uint64_t c = hist[t][bkt];
                hist[t][bkt] = acc;          // this thread's first slot in the bucket
                acc += c;
            }
        }
        bstart[NB] = acc;
    }
    std::vector<SeedRec> rec(rows);
    seed_parallel_ranges(rows, T, [&](unsigned t, uint64_t a, uint64_t b) {
        if (a >= b) return;
        uint64_t k = key_of(a);
        for (uint64_t p = a; p < b; p++) {
            SeedRec r;
            r.key = k;
            r.tie = tie_of(p);
            rec[hist[t][k >> 48]++] = r;
            k = (k << 2) | seed_code_at(w, L, p + kKeyBases);
        }
    });
    hist.clear();
    {
        std::atomic<uint32_t> next{0};
        std::vector<std::thread> th;
        for (unsigned t = 0; t < T; t++)
            th.emplace_back([&] {
                for (uint32_t bkt = next++; bkt < NB; bkt = next++)
                    std::sort(rec.begin() + bstart[bkt], rec.begin() + bstart[bkt + 1],
                              [](const SeedRec& x, const SeedRec& y) {
                                  return x.key != y.key ? x.key < y.key : x.tie < y.tie;
                              });
            });
        for (auto& x : th) x.join();
    }
    // 2. suffix array; BWT chunks: codes, then the counts before each chunk
    H.sa.assign(rows, 0);
    const uint64_t n_chunks = rows / kChunkRows + 1;
    H.occ.assign(n_chunks * 16, 0);
    std::vector<uint64_t> chunk_cnt(n_chunks * 4, 0);
    std::atomic<uint64_t> dollar{~0ull};
    seed_parallel_ranges(n_chunks, T, [&](unsigned, uint64_t a, uint64_t b) {
        for (uint64_t c = a; c < b; c++) {
            for (uint64_t i = c * kChunkRows; i < std::min(rows, (c + 1) * kChunkRows); i++) {
                const uint64_t p = seed_rec_pos(rec[i], L);
                H.sa[i] = (uint32_t)p;
                uint32_t b2 = 0;
                if (p == 0) {
                    dollar = i;
                } else {
                    b2 = seed_code_at(w, L, p - 1);
                    chunk_cnt[c * 4 + b2]++;
                }
                const uint64_t in = i - c * kChunkRows;
                H.occ[c * 16 + 4 + in / 32] |= (b2 & 1u) << (in % 32);         // low bit plane
                H.occ[c * 16 + 10 + in / 32] |= (b2 >> 1) << (in % 32);        // high bit plane
            }
        }
    });
    H.dollar_row = (uint32_t)dollar.load();
    uint64_t run[4] = {0, 0, 0, 0};
    for (uint64_t c = 0; c < n_chunks; c++)
        for (int b2 = 0; b2 < 4; b2++) {
            H.occ[c * 16 + b2] = (uint32_t)run[b2];
            run[b2] += chunk_cnt[c * 4 + b2];
        }
    H.C[0] = 1;
    for (int b2 = 1; b2 < 4; b2++) H.C[b2] = H.C[b2 - 1] + (uint32_t)run[b2 - 1];
    // 3. lookup table: rows whose first 12 bases are P form [lo, hi); the few
    // suffixes with fewer than 12 bases (X followed by the terminator) sort just
    // before the patterns they prefix, so they count below every P >= X.A...A
    std::vector<uint32_t> full(kLutSize, 0), shrt(kLutSize, 0);
    for (uint64_t i = 0; i < rows; i++) {
        const uint32_t P = (uint32_t)(rec[i].key >> (64 - 2 * kLutK));
        if (rec[i].tie >= (uint32_t)kLutK) full[P]++;
        else shrt[P]++;
    }
    H.lut.assign(kLutSize, RowInterval{0, 0});
    uint64_t below = 0, shorter = 0;
    for (uint32_t P = 0; P < kLutSize; P++) {
        shorter += shrt[P];
        const uint64_t lo = below + shorter;
        H.lut[P] = RowInterval{(uint32_t)lo, (uint32_t)(lo + full[P])};
        below += full[P];
    }
}

}  // namespace sa
