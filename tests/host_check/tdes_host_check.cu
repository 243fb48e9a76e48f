// Host-side run of the generated bitsliced and scalar 3DES code (test
// infrastructure only).  It compiles the very headers the kernels use, with
// their host versions of lop3 and byte_perm, so the generated circuits,
// key-table recipes and plane renames can be checked against the CPU oracle
// without a GPU.
//
// Usage: tdes_host_check <bs_enc|bs_dec|b1_enc|b1_dec|sc_enc|sc_dec|sn_enc|sn_dec|s1_enc|s1_dec>
//                        <48 hex K1||K2||K3>
//   reads whole 8-byte blocks on stdin, writes the results on stdout.
//   b1_*: the single-DES (one-pass) bitsliced tables and rounds under K1.
//   s1_*: the 16-round scalar round on the key words of (K1, K1, K1), as the
//         library builds them for a single-DES schedule.
//   mx_*: the mixed-key round (tdes_process32_mixed): block b of each group
//         of 32 is slot b, under the triple whose K1 has byte 0 XOR (2 * b).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_2007_10752_gb300/csrc/tdes_keysched.cuh"
#include "../../paper_2007_10752_gb300/csrc/tdes_scalar.cuh"
#include "../../paper_2007_10752_gb300/csrc/tdes_mixed.cuh"

static const uint8_t kRecipe[2][TDES_TABLE_WORDS][3] = TDES_RECIPE_INIT;
static const uint8_t kRecipe1[2][TDES1_TABLE_WORDS][3] = TDES1_RECIPE_INIT;
static const uint8_t kSub[2][48][48] = TDES_SUBKEY_INIT;
static const uint32_t kSP[8][64] = TDES_SP_INIT;
static const uint8_t kIP[64] = TDES_IP_INIT;
static const uint8_t kFP[64] = TDES_FP_INIT;
static const uint64_t kIPN[16][16] = TDES_IPN_INIT;
static const uint64_t kFPN[16][16] = TDES_FPN_INIT;

int main(int argc, char** argv) {
    if (argc != 3 || strlen(argv[2]) != 48) return 2;
    uint8_t keys[24];
    for (int i = 0; i < 24; ++i) {
        char h[3] = {argv[2][2 * i], argv[2][2 * i + 1], 0};
        keys[i] = (uint8_t)strtoul(h, nullptr, 16);
    }
    const bool dec = strstr(argv[1], "dec") != nullptr;
    if (strncmp(argv[1], "s1", 2) == 0) {  // a single-DES schedule holds (K1, K1, K1)
        memcpy(keys + 8, keys, 8);
        memcpy(keys + 16, keys, 8);
    }
    const bool bitsliced = argv[1][0] == 'b';
    const bool mixed = strncmp(argv[1], "mx", 2) == 0;
    const bool one_pass = strncmp(argv[1], "b1", 2) == 0;
    std::vector<uint8_t> data;
    uint8_t buf[1 << 16];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, stdin)) > 0) data.insert(data.end(), buf, buf + got);
    if (data.size() % 8) return 3;
    const size_t n = data.size() / 8;
    std::vector<uint8_t> out(data.size());

    if (mixed) {
        alignas(16) static uint32_t tab[TDES_TABLE_WORDS];
        for (int e = 0; e < TDES_TABLE_WORDS; ++e) {
            uint32_t w = 0;
            for (int sl = 0; sl < 32; ++sl) {
                uint8_t k[24];
                memcpy(k, keys, 24);
                k[0] ^= (uint8_t)(2 * sl);
                w |= (tdes_table_word(k, kRecipe[dec][e]) & 1u) << sl;
            }
            tab[e] = w;
        }
        for (size_t g0 = 0; g0 < n; g0 += 32) {
            uint32_t A0[32], A1[32];
            for (int sl = 0; sl < 32; ++sl) {
                uint32_t w[2] = {0, 0};
                if (g0 + sl < n) memcpy(w, &data[8 * (g0 + sl)], 8);
                A0[sl] = w[0];
                A1[sl] = w[1];
            }
            tdes_process32_mixed(A0, A1, tab);
            for (int sl = 0; sl < 32 && g0 + sl < n; ++sl) {
                uint32_t w[2] = {A0[sl], A1[sl]};
                memcpy(&out[8 * (g0 + sl)], w, 8);
            }
        }
    } else if (bitsliced) {
        alignas(16) static uint32_t tab[TDES_TABLE_WORDS];
        if (one_pass)
            for (int e = 0; e < TDES1_TABLE_WORDS; ++e) tab[e] = tdes_table_word(keys, kRecipe1[dec][e]);
        else
            for (int e = 0; e < TDES_TABLE_WORDS; ++e) tab[e] = tdes_table_word(keys, kRecipe[dec][e]);
        for (size_t g0 = 0; g0 < n; g0 += 32) {
            uint32_t A0[32], A1[32];
            for (int s = 0; s < 32; ++s) {
                uint32_t w[2] = {0, 0};
                if (g0 + s < n) memcpy(w, &data[8 * (g0 + s)], 8);
                A0[s] = w[0];
                A1[s] = w[1];
            }
            if (one_pass)
                tdes_process32<1>(A0, A1, tab);
            else
                tdes_process32<3>(A0, A1, tab);
            for (int s = 0; s < 32 && g0 + s < n; ++s) {
                uint32_t w[2] = {A0[s], A1[s]};
                memcpy(&out[8 * (g0 + s)], w, 8);
            }
        }
    } else {
        alignas(16) uint8_t chunks[TDES_SUBKEY_WORDS];
        for (int r = 0; r < 48; ++r)
            for (int g = 0; g < 8; ++g) chunks[8 * r + g] = tdes_subkey_chunk(keys, &kSub[dec][r][6 * g]);
        for (size_t i = 0; i < n; ++i) {
            uint64_t v;
            memcpy(&v, &data[8 * i], 8);
            v = bswap64(v);
            if (argv[1][1] == 'n')
                v = tdes_block_scalar_nib(v, &kSP[0][0], reinterpret_cast<const uint32_t*>(chunks),
                                          &kIPN[0][0], &kFPN[0][0]);
            else if (argv[1][1] == '1')
                v = tdes_block_scalar_nib<16>(v, &kSP[0][0],
                                              reinterpret_cast<const uint32_t*>(chunks),
                                              &kIPN[0][0], &kFPN[0][0]);
            else
                v = tdes_block_scalar(v, &kSP[0][0], reinterpret_cast<const uint32_t*>(chunks), kIP,
                                      kFP);
            v = bswap64(v);
            memcpy(&out[8 * i], &v, 8);
        }
    }
    fwrite(out.data(), 1, out.size(), stdout);
    return 0;
}
