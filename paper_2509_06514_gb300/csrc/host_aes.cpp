// host_aes.cpp — the product's host-side AES-128 pieces: the 32-bit T-table the GPU
// kernels expand into shared memory, the key schedule of the fixed MMO keys, and a
// T-table encryption used by the client-side key generator (dpf_gen).
//
// AES-128 is the PRF of Eq. (3) (§3.2, §4). Words are little-endian columns: word c of a
// block holds bytes 4c..4c+3 with byte 4c in bits 0..7.
#include <cstring>

#include "impir_internal.h"

namespace impir {
namespace {

struct Tables {
    uint8_t sbox[256];
    uint32_t te0[256];
    Tables() {
        // Powers of the generator {03} of GF(2^8)* and their logarithms.
        uint8_t expo[256], logt[256];
        uint8_t v = 1;
        for (int i = 0; i < 255; i++) {
            expo[i] = v;
            logt[v] = uint8_t(i);
            uint8_t dbl = uint8_t((v << 1) ^ ((v & 0x80) ? 0x1b : 0));
            v = uint8_t(v ^ dbl);  // v * {03}
        }
        logt[0] = 0;
        for (int x = 0; x < 256; x++) {
            uint8_t inv = x ? expo[(255 - logt[x]) % 255] : 0;
            // affine map: inv ^ rotl(inv,1) ^ rotl(inv,2) ^ rotl(inv,3) ^ rotl(inv,4) ^ {63}
            uint32_t r = inv;
            uint8_t s = uint8_t(r ^ ((r << 1) | (r >> 7)) ^ ((r << 2) | (r >> 6)) ^ ((r << 3) | (r >> 5)) ^
                                ((r << 4) | (r >> 4)) ^ 0x63);
            sbox[x] = s;
            uint8_t s2 = uint8_t((s << 1) ^ ((s & 0x80) ? 0x1b : 0));
            uint8_t s3 = uint8_t(s2 ^ s);
            // bytes (2S, S, S, 3S): column 0 of MixColumns applied to S
            te0[x] = uint32_t(s2) | (uint32_t(s) << 8) | (uint32_t(s) << 16) | (uint32_t(s3) << 24);
        }
    }
};

const Tables& tables() {
    static Tables t;
    return t;
}

inline uint32_t rotl32(uint32_t x, int n) { return (x << n) | (x >> (32 - n)); }
inline uint32_t tek(int k, uint32_t x) {
    uint32_t t = tables().te0[x & 0xff];
    return k == 0 ? t : rotl32(t, 8 * k);
}
inline uint32_t sb(uint32_t x) { return tables().sbox[x & 0xff]; }
inline uint32_t load_le(const uint8_t* p) {
    return uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16) | (uint32_t(p[3]) << 24);
}
inline void store_le(uint8_t* p, uint32_t v) {
    p[0] = uint8_t(v);
    p[1] = uint8_t(v >> 8);
    p[2] = uint8_t(v >> 16);
    p[3] = uint8_t(v >> 24);
}

}  // namespace

void host_aes_te0(uint32_t out[256]) { std::memcpy(out, tables().te0, sizeof(tables().te0)); }

void host_aes_expand(const uint8_t key[16], uint32_t rk[44]) {
    static const uint32_t rcon[10] = {0x01, 0x02, 0x04, 0x08, 0x10, 0x20, 0x40, 0x80, 0x1b, 0x36};
    for (int i = 0; i < 4; i++) rk[i] = load_le(key + 4 * i);
    for (int r = 1; r <= 10; r++) {
        uint32_t w = rk[4 * r - 1];
        // SubWord(RotWord(w)) on a little-endian word: byte b of the result is S(byte b+1)
        uint32_t t = sb(w >> 8) | (sb(w >> 16) << 8) | (sb(w >> 24) << 16) | (sb(w) << 24);
        rk[4 * r] = rk[4 * r - 4] ^ t ^ rcon[r - 1];
        rk[4 * r + 1] = rk[4 * r - 3] ^ rk[4 * r];
        rk[4 * r + 2] = rk[4 * r - 2] ^ rk[4 * r + 1];
        rk[4 * r + 3] = rk[4 * r - 1] ^ rk[4 * r + 2];
    }
}

void host_aes_encrypt(const uint32_t rk[44], const uint8_t in[16], uint8_t out[16]) {
    uint32_t s[4], n[4];
    for (int c = 0; c < 4; c++) s[c] = load_le(in + 4 * c) ^ rk[c];
    for (int r = 1; r < 10; r++) {
        for (int c = 0; c < 4; c++)
            n[c] = tek(0, s[c]) ^ tek(1, s[(c + 1) & 3] >> 8) ^ tek(2, s[(c + 2) & 3] >> 16) ^
                   tek(3, s[(c + 3) & 3] >> 24) ^ rk[4 * r + c];
        std::memcpy(s, n, sizeof(s));
    }
    for (int c = 0; c < 4; c++)
        n[c] = sb(s[c]) | (sb(s[(c + 1) & 3] >> 8) << 8) | (sb(s[(c + 2) & 3] >> 16) << 16) |
               (sb(s[(c + 3) & 3] >> 24) << 24);
    for (int c = 0; c < 4; c++) store_le(out + 4 * c, n[c] ^ rk[40 + c]);
}

}  // namespace impir
