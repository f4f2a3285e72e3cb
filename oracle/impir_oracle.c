/*
 * impir_oracle.c — plain, slow, obviously-correct CPU oracle for the server side of
 * two-server DPF-based PIR as defined in IM-PIR (arXiv 2509.06514).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library. It shares no code, header, table or constant
 * generator with the CUDA path; the product never links or calls it.
 *
 * What it computes, each function citing the passage it follows:
 *   - AES-128 (the PRF the paper uses, §3.2 and §4), written byte by byte from the
 *     AES standard (FIPS-197): S-box from the GF(2^8) inverse plus the affine map,
 *     KeyExpansion, SubBytes, ShiftRows, MixColumns (via xtime), AddRoundKey.
 *   - The PRF of Eq. (3): PRF_s(x) "encrypts x with key s" (§3.2): AES with key s over
 *     the block whose byte 0 is x and whose other bytes are zero. A second, fixed-key
 *     variant (Matyas-Meyer-Oseas) PRF_s(x) = AES_{K_x}(s) XOR s is offered too.
 *   - The GGM tree of Eqs. (1)-(3) (§3.2): R(0,0) = C_0[0,0];
 *     R(d,j) = PRF_{R(d-1,j>>1)}(j mod 2) XOR C_{R(d-1,j>>1) mod 2}[j mod 2, d];
 *     Eval(k,j) = R(m,j). Written twice: recursively (the branch-parallel reading,
 *     one root-to-leaf walk per leaf) and level by level (the level-by-level reading).
 *   - The selection bit v[j] = lsb(R(m,j)) and dpXOR r = XOR_{j : v[j]=1} D[j]
 *     (§2.3 and §3.3, Algorithm 1 TaskletXOR/MasterXOR/AggregateSubresults written as
 *     a single plain loop).
 *   - A key generator Gen(alpha) (§3.1 gives only its signature and the key shape; the
 *     construction here is the one that makes Eq. (3) hold for both keys) and the
 *     client reconstruction D[i] = r1 XOR r2 (§2.3).
 *   - A threaded answer that follows the paper's subtree split (§3.2: a master
 *     expands the tree down to level L, workers expand the 2^L perfect subtrees, then
 *     partial XORs are aggregated), used for the timed CPU baseline and for oracle
 *     checks of GB-scale databases.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   - "mod 2" of a 128-bit seed is bit 0 of byte 0 (little-endian field element).
 *   - "+" in Eq. (3) is XOR (addition in F_{2^lambda}).
 *   - enc(x) is the 16-byte block with byte 0 = x, other bytes 0.
 *   - The leaf's selection bit is the lsb of R(m,j).
 *   - Leaves j >= N select nothing; a key with 2^m < N covers the prefix [0, 2^m).
 *
 * Wire format of a key (little-endian), the format both sides parse independently:
 *   byte 0 version = 1, byte 1 prf (0 keyed, 1 MMO), byte 2 m (1..40), byte 3 the party
 *   index b (0 or 1; only the additive answer uses it), bytes 4..7 = 0, then
 *   C_0[2][m+1][16] and then C_1[2][m+1][16], where the first
 *   index is the child bit x (row), the second the depth d (column). Column 0 holds
 *   only the root seed C_0[0][0]; C_0[1][0], C_1[0][0], C_1[1][0] must be zero.
 *
 * Parity status: every function here is pinned by the non-GPU tests (FIPS-197 vectors
 * and a library AES, the two tree evaluation orders, brute-force DPF correctness, the
 * worked dpXOR example of Fig. 2, linearity, reconstruction).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------------------
 * AES-128, FIPS-197
 * ---------------------------------------------------------------------------------- */

/* Multiplication in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1 (FIPS-197 §4.2). */
static uint8_t gf_mul(uint8_t a, uint8_t b) {
    uint8_t p = 0;
    for (int i = 0; i < 8; i++) {
        if (b & 1) p ^= a;
        uint8_t hi = a & 0x80;
        a = (uint8_t)(a << 1);
        if (hi) a ^= 0x1b;
        b >>= 1;
    }
    return p;
}

/* xtime(a) = a * {02} (FIPS-197 §4.2.1). */
static uint8_t xtime(uint8_t a) { return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00)); }

static uint8_t SBOX[256];
static int sbox_ready = 0;

/* S-box (FIPS-197 §5.1.1): multiplicative inverse in GF(2^8) ({00} maps to {00}),
 * then the affine map b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i, c = {63}.
 * The inverse is found by exhaustive search, which is slow but plainly correct. */
static void build_sbox(void) {
    for (int x = 0; x < 256; x++) {
        uint8_t inv = 0;
        if (x != 0) {
            for (int y = 1; y < 256; y++) {
                if (gf_mul((uint8_t)x, (uint8_t)y) == 1) { inv = (uint8_t)y; break; }
            }
        }
        uint8_t s = 0;
        for (int i = 0; i < 8; i++) {
            int bit = ((inv >> i) & 1) ^ ((inv >> ((i + 4) % 8)) & 1) ^ ((inv >> ((i + 5) % 8)) & 1) ^
                      ((inv >> ((i + 6) % 8)) & 1) ^ ((inv >> ((i + 7) % 8)) & 1) ^ ((0x63 >> i) & 1);
            s |= (uint8_t)(bit << i);
        }
        SBOX[x] = s;
    }
    sbox_ready = 1;
}

static void ensure_sbox(void) {
    if (!sbox_ready) build_sbox();
}

/* KeyExpansion (FIPS-197 §5.2): 44 words w[i] of 4 bytes; round key r = w[4r..4r+3]. */
static void key_expansion(const uint8_t key[16], uint8_t w[44][4]) {
    static const uint8_t rcon[11] = {0x00, 0x01, 0x02, 0x04, 0x08, 0x10, 0x20, 0x40, 0x80, 0x1b, 0x36};
    for (int i = 0; i < 4; i++)
        for (int b = 0; b < 4; b++) w[i][b] = key[4 * i + b];
    for (int i = 4; i < 44; i++) {
        uint8_t temp[4];
        memcpy(temp, w[i - 1], 4);
        if (i % 4 == 0) {
            /* RotWord then SubWord then XOR Rcon[i/4] */
            uint8_t t0 = temp[0];
            temp[0] = temp[1];
            temp[1] = temp[2];
            temp[2] = temp[3];
            temp[3] = t0;
            for (int b = 0; b < 4; b++) temp[b] = SBOX[temp[b]];
            temp[0] ^= rcon[i / 4];
        }
        for (int b = 0; b < 4; b++) w[i][b] = w[i - 4][b] ^ temp[b];
    }
}

/* Cipher (FIPS-197 §5.1) with state[r][c] = in[r + 4c]. */
static void cipher(const uint8_t w[44][4], const uint8_t in[16], uint8_t out[16]) {
    uint8_t st[4][4];
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) st[r][c] = in[r + 4 * c];
    /* AddRoundKey(round 0) */
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) st[r][c] ^= w[c][r];
    for (int round = 1; round <= 10; round++) {
        /* SubBytes */
        for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++) st[r][c] = SBOX[st[r][c]];
        /* ShiftRows: row r rotates left by r */
        for (int r = 1; r < 4; r++) {
            uint8_t tmp[4];
            for (int c = 0; c < 4; c++) tmp[c] = st[r][(c + r) % 4];
            for (int c = 0; c < 4; c++) st[r][c] = tmp[c];
        }
        /* MixColumns (skipped in the final round) */
        if (round != 10) {
            for (int c = 0; c < 4; c++) {
                uint8_t a0 = st[0][c], a1 = st[1][c], a2 = st[2][c], a3 = st[3][c];
                /* {02}a0 ^ {03}a1 ^ a2 ^ a3, {03}a = xtime(a) ^ a */
                st[0][c] = (uint8_t)(xtime(a0) ^ (xtime(a1) ^ a1) ^ a2 ^ a3);
                st[1][c] = (uint8_t)(a0 ^ xtime(a1) ^ (xtime(a2) ^ a2) ^ a3);
                st[2][c] = (uint8_t)(a0 ^ a1 ^ xtime(a2) ^ (xtime(a3) ^ a3));
                st[3][c] = (uint8_t)((xtime(a0) ^ a0) ^ a1 ^ a2 ^ xtime(a3));
            }
        }
        /* AddRoundKey */
        for (int c = 0; c < 4; c++)
            for (int r = 0; r < 4; r++) st[r][c] ^= w[4 * round + c][r];
    }
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) out[r + 4 * c] = st[r][c];
}

void orc_aes128_encrypt(const uint8_t key[16], const uint8_t in[16], uint8_t out[16]) {
    ensure_sbox();
    uint8_t w[44][4];
    key_expansion(key, w);
    cipher(w, in, out);
}

/* Round keys exposed for the key-expansion test (176 bytes, round key r at 16r). */
void orc_aes128_round_keys(const uint8_t key[16], uint8_t rk[176]) {
    ensure_sbox();
    uint8_t w[44][4];
    key_expansion(key, w);
    for (int i = 0; i < 44; i++)
        for (int b = 0; b < 4; b++) rk[4 * i + b] = w[i][b];
}

uint8_t orc_sbox(uint8_t x) {
    ensure_sbox();
    return SBOX[x];
}

/* ------------------------------------------------------------------------------------
 * PRF (§3.2, §4): AES-128
 * ---------------------------------------------------------------------------------- */

/* The two fixed keys of the Matyas-Meyer-Oseas variant (a project choice; the paper's
 * own PRF is the keyed one). ASCII "IM-PIR MMO key 0" and "IM-PIR MMO key 1". */
static const uint8_t MMO_KEY[2][16] = {
    {'I', 'M', '-', 'P', 'I', 'R', ' ', 'M', 'M', 'O', ' ', 'k', 'e', 'y', ' ', '0'},
    {'I', 'M', '-', 'P', 'I', 'R', ' ', 'M', 'M', 'O', ' ', 'k', 'e', 'y', ' ', '1'},
};

/* PRF_s(x) for x in {0, 1}.
 * prf = 0: "encrypts a value x with an encryption key s" (§3.2): AES_s(enc(x)).
 * prf = 1: AES_{K_x}(s) XOR s. */
void orc_prf(int prf, const uint8_t s[16], int x, uint8_t out[16]) {
    if (prf == 0) {
        uint8_t blk[16] = {0};
        blk[0] = (uint8_t)x;
        orc_aes128_encrypt(s, blk, out);
    } else {
        uint8_t e[16];
        orc_aes128_encrypt(MMO_KEY[x], s, e);
        for (int i = 0; i < 16; i++) out[i] = e[i] ^ s[i];
    }
}

/* ------------------------------------------------------------------------------------
 * DPF keys (§3.1): two codewords C_0, C_1 in F_{2^128}^{2 x (m+1)}
 * ---------------------------------------------------------------------------------- */

typedef struct {
    uint32_t m;
    int prf;
    int party;           /* header byte 3 */
    const uint8_t* C[2]; /* C[t] points at C_t[2][m+1][16] inside the wire key */
} orc_key;

size_t orc_key_bytes(uint32_t m) { return 8 + (size_t)64 * (m + 1); }

static const uint8_t* cw(const orc_key* k, int t, int x, uint32_t d) {
    return k->C[t] + ((size_t)x * (k->m + 1) + d) * 16;
}

/* Parses and validates one wire key. Returns 0 on success. */
static int parse_key(const uint8_t* buf, orc_key* k) {
    if (buf[0] != 1) return ORC_EINVAL;
    if (buf[1] > 1) return ORC_EINVAL;
    if (buf[2] < 1 || buf[2] > 40) return ORC_EINVAL;
    if (buf[3] > 1 || buf[4] != 0 || buf[5] != 0 || buf[6] != 0 || buf[7] != 0) return ORC_EINVAL;
    k->m = buf[2];
    k->prf = buf[1];
    k->party = buf[3];
    k->C[0] = buf + 8;
    k->C[1] = buf + 8 + (size_t)32 * (k->m + 1);
    /* column 0 holds only the root C_0[0][0] */
    const uint8_t* z[3] = {cw(k, 0, 1, 0), cw(k, 1, 0, 0), cw(k, 1, 1, 0)};
    for (int i = 0; i < 3; i++)
        for (int b = 0; b < 16; b++)
            if (z[i][b]) return ORC_EINVAL;
    return ORC_OK;
}

int orc_key_check(const uint8_t* key) {
    orc_key k;
    return parse_key(key, &k);
}

/* One edge of the tree, Eq. (3): child x of parent p at depth d. */
static void child(const orc_key* k, const uint8_t p[16], int x, uint32_t d, uint8_t out[16]) {
    int t = p[0] & 1; /* "R(d-1, j/2) mod 2" */
    uint8_t f[16];
    orc_prf(k->prf, p, x, f);
    const uint8_t* c = cw(k, t, x, d);
    for (int i = 0; i < 16; i++) out[i] = f[i] ^ c[i];
}

/* R(d, j) written as the recursion of Eqs. (2)-(3): the branch-parallel reading. */
static void node_value(const orc_key* k, uint32_t d, uint64_t j, uint8_t out[16]) {
    if (d == 0) { /* Eq. (2) */
        memcpy(out, cw(k, 0, 0, 0), 16);
        return;
    }
    uint8_t parent[16];
    node_value(k, d - 1, j >> 1, parent);
    child(k, parent, (int)(j & 1), d, out);
}

/* Eval(k, j) = R(m, j), Eq. (1): the full 128-bit leaf. */
int orc_eval_point(const uint8_t* key, uint64_t j, uint8_t out[16]) {
    orc_key k;
    int rc = parse_key(key, &k);
    if (rc) return rc;
    if (k.m < 64 && (j >> k.m) != 0) return ORC_EINVAL;
    ensure_sbox();
    node_value(&k, k.m, j, out);
    return ORC_OK;
}

/* Level-by-level expansion of the subtree under node (d0, j0) down to depth d0 + h:
 * every level fully materialised (the level-by-level reading of §3.2). Writes
 * 2^h leaves of 16 bytes to out; scratch needs 2^h * 16 bytes. */
static void expand_levels(const orc_key* k, uint32_t d0, const uint8_t root[16], uint32_t h, uint8_t* out,
                          uint8_t* scratch) {
    /* the final level must land in out: alternate so that level h is in out */
    uint8_t* bufs[2];
    bufs[h % 2] = out;
    bufs[(h + 1) % 2] = scratch;
    memcpy(bufs[0], root, 16);
    for (uint32_t l = 0; l < h; l++) {
        uint8_t* cur = bufs[l % 2];
        uint8_t* nxt = bufs[(l + 1) % 2];
        uint64_t n = (uint64_t)1 << l;
        /* go from the end so in-place aliasing never matters (buffers differ anyway) */
        for (uint64_t i = 0; i < n; i++) {
            child(k, cur + 16 * i, 0, d0 + l + 1, nxt + 16 * (2 * i));
            child(k, cur + 16 * i, 1, d0 + l + 1, nxt + 16 * (2 * i + 1));
        }
    }
}

/* EvalAll: all 2^m leaves, level by level (m <= 26 here: 1 GiB of leaves). */
int orc_eval_all(const uint8_t* key, uint8_t* leaves) {
    orc_key k;
    int rc = parse_key(key, &k);
    if (rc) return rc;
    if (k.m > 26) return ORC_EINVAL;
    ensure_sbox();
    uint8_t* scratch = (uint8_t*)malloc(((size_t)1 << k.m) * 16);
    if (!scratch) return ORC_ENOMEM;
    expand_levels(&k, 0, cw(&k, 0, 0, 0), k.m, leaves, scratch);
    free(scratch);
    return ORC_OK;
}

/* The function-share bit vector v[j] = lsb(Eval(k, j)) for j < n (n <= 2^m). */
int orc_eval_bits(const uint8_t* key, uint64_t n, uint8_t* bits) {
    orc_key k;
    int rc = parse_key(key, &k);
    if (rc) return rc;
    if (k.m > 26 || n > ((uint64_t)1 << k.m)) return ORC_EINVAL;
    uint8_t* leaves = (uint8_t*)malloc(((size_t)1 << k.m) * 16);
    if (!leaves) return ORC_ENOMEM;
    rc = orc_eval_all(key, leaves);
    if (rc == ORC_OK)
        for (uint64_t j = 0; j < n; j++) bits[j] = leaves[16 * j] & 1;
    free(leaves);
    return rc;
}

/* dpXOR (§2.3, §3.3): out = XOR of D[j] over j < n with bits[j] = 1. */
void orc_dpxor(const uint8_t* db, uint64_t n, uint32_t record_bytes, const uint8_t* bits, uint8_t* out) {
    memset(out, 0, record_bytes);
    for (uint64_t j = 0; j < n; j++) {
        if (bits[j] & 1) {
            const uint8_t* rec = db + j * (uint64_t)record_bytes;
            for (uint32_t b = 0; b < record_bytes; b++) out[b] ^= rec[b];
        }
    }
}

/* One server's answer: r = XOR_{j < min(N, 2^m)} v[j] * D[j]. Single-threaded. */
int orc_answer(const uint8_t* key, const uint8_t* db, uint64_t N, uint32_t record_bytes, uint8_t* out) {
    orc_key k;
    int rc = parse_key(key, &k);
    if (rc) return rc;
    if (record_bytes == 0 || N == 0) return ORC_EINVAL;
    if (k.m > 26) return ORC_EINVAL;
    uint64_t dom = (uint64_t)1 << k.m;
    uint64_t n = N < dom ? N : dom;
    uint8_t* bits = (uint8_t*)malloc(dom);
    if (!bits) return ORC_ENOMEM;
    rc = orc_eval_bits(key, dom, bits);
    if (rc == ORC_OK) orc_dpxor(db, n, record_bytes, bits, out);
    free(bits);
    return rc;
}

/* One server's answer with every leaf evaluated on its own root-to-leaf walk (the
 * branch-parallel reading of §3.2): for any domain size, cost m AES per record covered. */
int orc_answer_points(const uint8_t* key, const uint8_t* db, uint64_t N, uint32_t record_bytes, uint8_t* out) {
    orc_key k;
    int rc = parse_key(key, &k);
    if (rc) return rc;
    if (record_bytes == 0 || N == 0) return ORC_EINVAL;
    ensure_sbox();
    uint64_t dom = k.m >= 64 ? UINT64_MAX : ((uint64_t)1 << k.m);
    uint64_t n = N < dom ? N : dom;
    memset(out, 0, record_bytes);
    for (uint64_t j = 0; j < n; j++) {
        uint8_t leaf[16];
        node_value(&k, k.m, j, leaf);
        if (leaf[0] & 1) {
            const uint8_t* rec = db + j * (uint64_t)record_bytes;
            for (uint32_t b = 0; b < record_bytes; b++) out[b] ^= rec[b];
        }
    }
    return ORC_OK;
}

/* The additive (inner-product) answer of §2.2 over Z_{2^32}: records are vectors of
 * little-endian 32-bit words and server b returns r_b = sum_j v_b[j] * D[j] (mod 2^32, word
 * by word) with the share v_b[j] = (-1)^b * low32(R(m,j)), low32 being bytes 0..3 of the leaf
 * read little-endian and b the key's party index. Leaves of the two keys agree off the point
 * and differ by the integer 1 at it, so the shares sum to 0 off the point and, because Gen
 * makes lsb(R_0(m, alpha)) = 1, to +1 at it: r_0 + r_1 = D[alpha]. record_bytes must be a
 * multiple of 4. Every leaf on its own root-to-leaf walk, for any domain size. */
int orc_answer_add32(const uint8_t* key, const uint8_t* db, uint64_t N, uint32_t record_bytes, uint8_t* out) {
    orc_key k;
    int rc = parse_key(key, &k);
    if (rc) return rc;
    if (record_bytes == 0 || record_bytes % 4 || N == 0) return ORC_EINVAL;
    ensure_sbox();
    uint64_t dom = k.m >= 64 ? UINT64_MAX : ((uint64_t)1 << k.m);
    uint64_t n = N < dom ? N : dom;
    uint32_t words = record_bytes / 4;
    uint32_t* acc = (uint32_t*)calloc(words, sizeof(uint32_t));
    if (!acc) return ORC_ENOMEM;
    for (uint64_t j = 0; j < n; j++) {
        uint8_t leaf[16];
        node_value(&k, k.m, j, leaf);
        uint32_t v = (uint32_t)leaf[0] | ((uint32_t)leaf[1] << 8) | ((uint32_t)leaf[2] << 16) | ((uint32_t)leaf[3] << 24);
        if (k.party) v = 0u - v;
        const uint8_t* rec = db + j * (uint64_t)record_bytes;
        for (uint32_t w = 0; w < words; w++) {
            uint32_t d = (uint32_t)rec[4 * w] | ((uint32_t)rec[4 * w + 1] << 8) | ((uint32_t)rec[4 * w + 2] << 16) |
                         ((uint32_t)rec[4 * w + 3] << 24);
            acc[w] += v * d;
        }
    }
    for (uint32_t w = 0; w < words; w++)
        for (int b = 0; b < 4; b++) out[4 * w + b] = (uint8_t)(acc[w] >> (8 * b));
    free(acc);
    return ORC_OK;
}

/* D[i] = r_0 + r_1 (mod 2^32, word by word): the client side of the additive answer. */
void orc_reconstruct_add32(const uint8_t* r0, const uint8_t* r1, uint32_t record_bytes, uint8_t* out) {
    for (uint32_t w = 0; w + 4 <= record_bytes; w += 4) {
        uint32_t a = 0, b = 0;
        for (int i = 0; i < 4; i++) {
            a |= (uint32_t)r0[w + i] << (8 * i);
            b |= (uint32_t)r1[w + i] << (8 * i);
        }
        uint32_t c = a + b;
        for (int i = 0; i < 4; i++) out[w + i] = (uint8_t)(c >> (8 * i));
    }
}

/* ------------------------------------------------------------------------------------
 * Threaded answer: the paper's subtree split (§3.2) + two-stage reduction (§3.3)
 * ---------------------------------------------------------------------------------- */

typedef struct {
    const orc_key* k;
    const uint8_t* db;
    uint64_t n;         /* records covered: min(N, 2^m) */
    uint32_t B;
    uint32_t L;         /* split level */
    const uint8_t* top; /* 2^L nodes at depth L */
    uint64_t next;      /* next subtree to take (guarded by mu) */
    pthread_mutex_t mu;
} par_job;

typedef struct {
    par_job* job;
    uint8_t* partial; /* this worker's partial XOR t_i */
    int rc;
} par_worker;

static void* par_run(void* arg) {
    par_worker* w = (par_worker*)arg;
    par_job* J = w->job;
    uint32_t h = J->k->m - J->L;
    uint64_t leaves = (uint64_t)1 << h;
    uint8_t* buf = (uint8_t*)malloc(leaves * 16);
    uint8_t* scratch = (uint8_t*)malloc(leaves * 16);
    if (!buf || !scratch) {
        w->rc = ORC_ENOMEM;
        free(buf);
        free(scratch);
        return NULL;
    }
    memset(w->partial, 0, J->B);
    for (;;) {
        pthread_mutex_lock(&J->mu);
        uint64_t s = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (s >= ((uint64_t)1 << J->L)) break;
        uint64_t base = s << h;
        if (base >= J->n) continue; /* subtree entirely beyond the database */
        expand_levels(J->k, J->L, J->top + 16 * s, h, buf, scratch);
        for (uint64_t i = 0; i < leaves && base + i < J->n; i++) {
            if (buf[16 * i] & 1) {
                const uint8_t* rec = J->db + (base + i) * (uint64_t)J->B;
                for (uint32_t b = 0; b < J->B; b++) w->partial[b] ^= rec[b];
            }
        }
    }
    free(buf);
    free(scratch);
    w->rc = ORC_OK;
    return NULL;
}

/* Same result as orc_answer, computed by a master that expands the tree to level L and
 * nthreads workers that each take whole perfect subtrees of depth m - L (§3.2), then the
 * partial XORs are combined (§3.3, Algorithm 1). */
int orc_answer_threads(const uint8_t* key, const uint8_t* db, uint64_t N, uint32_t record_bytes, uint8_t* out,
                       int nthreads) {
    orc_key k;
    int rc = parse_key(key, &k);
    if (rc) return rc;
    if (record_bytes == 0 || N == 0 || nthreads < 1) return ORC_EINVAL;
    ensure_sbox();
    uint64_t dom = k.m >= 64 ? UINT64_MAX : ((uint64_t)1 << k.m);
    uint64_t n = N < dom ? N : dom;
    /* enough subtrees to balance the workers; each subtree at most 2^22 leaves */
    uint32_t L = 0;
    while (((uint64_t)1 << L) < (uint64_t)nthreads * 8 && L < k.m) L++;
    while (k.m - L > 22) L++;
    if (L > 30) return ORC_EINVAL;
    uint8_t* top = (uint8_t*)malloc(((size_t)1 << L) * 16);
    uint8_t* scratch = (uint8_t*)malloc(((size_t)1 << L) * 16);
    par_worker* ws = (par_worker*)calloc((size_t)nthreads, sizeof(par_worker));
    uint8_t* partials = (uint8_t*)malloc((size_t)nthreads * record_bytes);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!top || !scratch || !ws || !partials || !th) {
        free(top);
        free(scratch);
        free(ws);
        free(partials);
        free(th);
        return ORC_ENOMEM;
    }
    expand_levels(&k, 0, cw(&k, 0, 0, 0), L, top, scratch); /* master: root to level L */
    par_job J;
    J.k = &k;
    J.db = db;
    J.n = n;
    J.B = record_bytes;
    J.L = L;
    J.top = top;
    J.next = 0;
    pthread_mutex_init(&J.mu, NULL);
    for (int i = 0; i < nthreads; i++) {
        ws[i].job = &J;
        ws[i].partial = partials + (size_t)i * record_bytes;
        ws[i].rc = ORC_OK;
        pthread_create(&th[i], NULL, par_run, &ws[i]);
    }
    memset(out, 0, record_bytes);
    rc = ORC_OK;
    for (int i = 0; i < nthreads; i++) {
        pthread_join(th[i], NULL);
        if (ws[i].rc) rc = ws[i].rc;
        for (uint32_t b = 0; b < record_bytes; b++) out[b] ^= ws[i].partial[b]; /* aggregate */
    }
    pthread_mutex_destroy(&J.mu);
    free(top);
    free(scratch);
    free(ws);
    free(partials);
    free(th);
    return rc;
}

/* ------------------------------------------------------------------------------------
 * Client side: Gen and reconstruction
 * ---------------------------------------------------------------------------------- */

/* SplitMix64 (Steele, Lea and Flood, 2014): the generator both key generators draw
 * from, seeded by the XOR of the four little-endian 64-bit words of the 32-byte seed. */
typedef struct {
    uint64_t x;
} sm64;

static uint64_t sm64_next(sm64* g) {
    uint64_t z = (g->x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void sm64_block(sm64* g, uint8_t out[16]) {
    for (int h = 0; h < 2; h++) {
        uint64_t v = sm64_next(g);
        for (int b = 0; b < 8; b++) out[8 * h + b] = (uint8_t)(v >> (8 * b));
    }
}

/* Gen(alpha) -> (key0, key1) with Eval(key0,j) XOR Eval(key1,j) = [j == alpha] as 128-bit
 * values for every j < 2^m (the DPF property of §2.3 with b = 1).
 * Draw order: s_A, s_B; then for d = 1..m and x = 0, 1: a uniform r, and, when x is the
 * on-path bit and d < m, a uniform delta with lsb forced to 1. At the leaf on the path the
 * lsb of r is then set so that lsb(R_A(m, alpha)) = 1, which makes the additive shares of
 * the two parties (key0 party 0, key1 party 1) sum to +1 rather than -1 at alpha. */
int orc_gen(uint64_t alpha, uint32_t m, int prf, const uint8_t seed[32], uint8_t* key0, uint8_t* key1) {
    if (m < 1 || m > 40 || (prf != 0 && prf != 1)) return ORC_EINVAL;
    if ((alpha >> m) != 0) return ORC_EINVAL;
    ensure_sbox();
    sm64 g;
    g.x = 0;
    for (int w = 0; w < 4; w++) {
        uint64_t v = 0;
        for (int b = 0; b < 8; b++) v |= (uint64_t)seed[8 * w + b] << (8 * b);
        g.x ^= v;
    }
    size_t kb = orc_key_bytes(m);
    uint8_t* keys[2] = {key0, key1};
    for (int i = 0; i < 2; i++) {
        memset(keys[i], 0, kb);
        keys[i][0] = 1;
        keys[i][1] = (uint8_t)prf;
        keys[i][2] = (uint8_t)m;
        keys[i][3] = (uint8_t)i; /* party index */
    }
    /* C_t[x][d] lives at 8 + t*32*(m+1) + (x*(m+1) + d)*16, identical in both keys for d >= 1 */
#define ORC_CW(key, t, x, d) ((key) + 8 + (size_t)(t) * 32 * (m + 1) + ((size_t)(x) * (m + 1) + (d)) * 16)
    uint8_t pA[16], pB[16];
    sm64_block(&g, pA);
    sm64_block(&g, pB);
    pB[0] = (uint8_t)((pB[0] & 0xfe) | ((pA[0] & 1) ^ 1)); /* control bits differ at the root */
    memcpy(ORC_CW(key0, 0, 0, 0), pA, 16);
    memcpy(ORC_CW(key1, 0, 0, 0), pB, 16);
    for (uint32_t d = 1; d <= m; d++) {
        int a = pA[0] & 1; /* key A's parent uses C_a, key B's uses C_{1-a} */
        int ad = (int)((alpha >> (m - d)) & 1);
        uint8_t fA[2][16], fB[2][16];
        for (int x = 0; x < 2; x++) {
            orc_prf(prf, pA, x, fA[x]);
            orc_prf(prf, pB, x, fB[x]);
            uint8_t r[16], delta[16] = {0};
            sm64_block(&g, r);
            if (d == m && x == ad) r[0] = (uint8_t)((r[0] & 0xfe) | ((fA[x][0] & 1) ^ 1)); /* lsb(R_A) = 1 */
            if (x == ad) {
                if (d < m) {
                    sm64_block(&g, delta);
                    delta[0] |= 1;
                } else {
                    delta[0] = 1; /* b = 1: the leaves differ by the integer 1 */
                }
            }
            uint8_t* ca = ORC_CW(key0, a, x, d);
            uint8_t* cb = ORC_CW(key0, 1 - a, x, d);
            for (int b = 0; b < 16; b++) {
                ca[b] = r[b];
                cb[b] = (uint8_t)(r[b] ^ fA[x][b] ^ fB[x][b] ^ delta[b]);
            }
        }
        /* columns d of both codewords are shared */
        for (int t = 0; t < 2; t++)
            for (int x = 0; x < 2; x++) memcpy(ORC_CW(key1, t, x, d), ORC_CW(key0, t, x, d), 16);
        uint8_t nA[16], nB[16];
        const uint8_t* ca = ORC_CW(key0, a, ad, d);
        const uint8_t* cb = ORC_CW(key0, 1 - a, ad, d);
        for (int b = 0; b < 16; b++) {
            nA[b] = fA[ad][b] ^ ca[b];
            nB[b] = fB[ad][b] ^ cb[b];
        }
        memcpy(pA, nA, 16);
        memcpy(pB, nB, 16);
    }
#undef ORC_CW
    return ORC_OK;
}

/* D[i] = r1 XOR r2 (§2.3). */
void orc_reconstruct(const uint8_t* r0, const uint8_t* r1, uint32_t record_bytes, uint8_t* out) {
    for (uint32_t b = 0; b < record_bytes; b++) out[b] = r0[b] ^ r1[b];
}

/* Number of AES-128 encryptions one full-domain evaluation performs: 2 (2^m - 1). */
uint64_t orc_aes_per_eval(uint32_t m) { return 2 * (((uint64_t)1 << m) - 1); }
