// Checks the seeding front end's host index (csrc/seed_index.h) against plain
// definitions on small references, without a GPU:
//  - the row order is the order of the suffixes (terminator smaller than every
//    base) compared on their first 32 bases, equal prefixes by position;
//  - every lookup-table interval holds exactly the rows that start with its
//    12-base pattern;
//  - backward search with the chunked BWT counts, started from the lookup
//    table, finds exactly the positions a direct scan finds.
// Usage: seed_index_check <length> <seed> <alphabet 2|4>; prints "ok" or the
// first difference and exits non-zero.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "seed_index.h"

static const char* B = "ACGT";

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    const uint64_t L = std::strtoull(argv[1], nullptr, 10);
    std::mt19937_64 rng(std::strtoull(argv[2], nullptr, 10));
    const int alpha = std::atoi(argv[3]);
    std::string s(L, 'A');
    for (auto& c : s) c = B[rng() % alpha];
    // plant a run and a repeat so that equal 32-base prefixes occur
    if (L > 400) {
        for (int i = 100; i < 160; i++) s[i] = 'A';
        for (int i = 0; i < 50; i++) s[300 + i] = s[200 + i];
    }
    std::vector<uint32_t> w((L + 15) / 16 + 4, 0);
    for (uint64_t p = 0; p < L; p++) {
        const uint32_t c = s[p] == 'A' ? 0 : s[p] == 'C' ? 1 : s[p] == 'G' ? 2 : 3;
        w[p >> 4] |= c << (2 * (p & 15));
    }
    sa::SeedHostIndex H;
    sa::build_seed_index(w.data(), L, H);
    const uint64_t rows = L + 1;
    // 1. row order: suffixes compared on up to 32 bases, the shorter one first
    //    when one prefixes the other within 32, then by position
    auto less_row = [&](uint64_t p, uint64_t q) {
        const std::string a = s.substr(p, 32), b = s.substr(q, 32);
        if (a != b) return a < b;      // std::string: a proper prefix compares smaller
        return p < q;
    };
    if (H.sa.size() != rows) { std::printf("sa size %zu\n", H.sa.size()); return 1; }
    for (uint64_t i = 0; i + 1 < rows; i++)
        if (!less_row(H.sa[i], H.sa[i + 1])) {
            std::printf("rows %llu, %llu out of order\n", (unsigned long long)i, (unsigned long long)i + 1);
            return 1;
        }
    // 2. lookup table
    std::vector<sa::RowInterval> want(sa::kLutSize, sa::RowInterval{0, 0});
    {
        // rows with >= 12 bases grouped by pattern; an empty pattern's interval is
        // empty at the first row that sorts after it
        std::vector<uint32_t> cnt(sa::kLutSize, 0);
        for (uint64_t i = 0; i < rows; i++) {
            const uint64_t p = H.sa[i];
            if (L - p < 12) continue;
            uint32_t P = 0;
            for (int t = 0; t < 12; t++) P = (P << 2) | (uint32_t)(std::string(B).find(s[p + t]));
            if (cnt[P] == 0) want[P].lo = (uint32_t)i;
            cnt[P]++;
            want[P].hi = (uint32_t)i + 1;
            if (want[P].hi - want[P].lo != cnt[P]) { std::printf("pattern %u rows not contiguous\n", P); return 1; }
        }
        // empty patterns: lo = hi = number of suffixes that sort before the pattern
        for (uint32_t P = 0; P < sa::kLutSize; P++) {
            if (cnt[P]) continue;
            std::string pat(12, 'A');
            for (int t = 0; t < 12; t++) pat[t] = B[(P >> (2 * (11 - t))) & 3];
            // binary search on the row order with the pattern as a 12-base key
            uint64_t lo = 0, hi = rows;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) / 2;
                if (s.substr(H.sa[mid], 12) < pat) lo = mid + 1; else hi = mid;
            }
            want[P].lo = want[P].hi = (uint32_t)lo;
        }
    }
    for (uint32_t P = 0; P < sa::kLutSize; P++)
        if (want[P].lo != H.lut[P].lo || want[P].hi != H.lut[P].hi) {
            std::printf("lut[%u] = [%u, %u), want [%u, %u)\n", P, H.lut[P].lo, H.lut[P].hi, want[P].lo, want[P].hi);
            return 1;
        }
    // 3. backward search from the lookup table with the chunked counts
    auto rank = [&](uint32_t i, uint32_t c) {
        const uint32_t chunk = i / sa::kChunkRows, in = i - chunk * sa::kChunkRows;
        uint32_t r = H.occ[chunk * 16 + c];
        for (uint32_t k = 0; k < in; k++) {
            const uint32_t e = ((H.occ[chunk * 16 + 4 + k / 32] >> (k % 32)) & 1u) |
                               (((H.occ[chunk * 16 + 10 + k / 32] >> (k % 32)) & 1u) << 1);
            const uint32_t row = chunk * sa::kChunkRows + k;
            if (e == c && row != H.dollar_row) r++;
        }
        return r;
    };
    for (int trial = 0; trial < 3000; trial++) {
        const int m = 12 + (int)(rng() % 21);
        std::string pat;
        if (trial % 3 && L > (uint64_t)m) pat = s.substr(rng() % (L - m + 1), m);
        else { pat.resize(m); for (auto& c : pat) c = B[rng() % alpha]; }
        uint32_t P = 0;
        for (int t = m - 12; t < m; t++) P = (P << 2) | (uint32_t)std::string(B).find(pat[t]);
        uint32_t lo = H.lut[P].lo, hi = H.lut[P].hi;
        for (int j = m - 13; j >= 0 && lo < hi; j--) {
            const uint32_t c = (uint32_t)std::string(B).find(pat[j]);
            lo = H.C[c] + rank(lo, c);
            hi = H.C[c] + rank(hi, c);
        }
        std::vector<uint64_t> got;
        for (uint32_t i = lo; i < hi; i++) got.push_back(H.sa[i]);
        std::sort(got.begin(), got.end());
        std::vector<uint64_t> want_pos;
        for (uint64_t p = 0; p + m <= L; p++)
            if (s.compare(p, m, pat) == 0) want_pos.push_back(p);
        if (got != want_pos) {
            std::printf("pattern %s: %zu positions found, %zu by scanning\n", pat.c_str(), got.size(), want_pos.size());
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
