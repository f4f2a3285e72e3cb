/*
 * inputs_gen.c — seeded synthetic input bytes for databases.
 *
 * Holds none of the PIR method's arithmetic: it only produces the uniform random record
 * bytes that both the CUDA path and the CPU oracle consume. Byte o of stream `seed` is
 * byte (o mod 8), little-endian, of the SplitMix64 output number o/8 for a generator whose
 * initial state is `seed` (Steele, Lea and Flood 2014): out_i = mix(seed + (i+1) * gamma).
 * Being counter-based, any byte range can be produced independently, so the fill is split
 * across threads and sampled records can be regenerated on their own.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Writes bytes [offset, offset + n) of stream `seed` to out. */
static void fill_range(uint8_t* out, uint64_t n, uint64_t seed, uint64_t offset) {
    uint64_t o = offset, end = offset + n;
    while (o < end && (o & 7)) {
        out[o - offset] = (uint8_t)(sm64_at(seed, o >> 3) >> (8 * (o & 7)));
        o++;
    }
    while (o + 8 <= end) {
        uint64_t v = sm64_at(seed, o >> 3);
        memcpy(out + (o - offset), &v, 8); /* little-endian hosts only (x86_64, aarch64) */
        o += 8;
    }
    while (o < end) {
        out[o - offset] = (uint8_t)(sm64_at(seed, o >> 3) >> (8 * (o & 7)));
        o++;
    }
}

typedef struct {
    uint8_t* out;
    uint64_t n, seed, offset;
} fill_job;

static void* fill_thread(void* a) {
    fill_job* j = (fill_job*)a;
    fill_range(j->out, j->n, j->seed, j->offset);
    return NULL;
}

int impir_inputs_fill(uint8_t* out, uint64_t n, uint64_t seed, uint64_t offset, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (n < (1u << 20) || threads == 1) {
        fill_range(out, n, seed, offset);
        return 0;
    }
    pthread_t th[256];
    int joined[256];
    fill_job jobs[256];
    uint64_t chunk = ((n / (uint64_t)threads) + 7) & ~(uint64_t)7;
    int used = 0;
    for (int t = 0; t < threads; t++) {
        uint64_t lo = (uint64_t)t * chunk;
        if (lo >= n) break;
        uint64_t hi = lo + chunk < n ? lo + chunk : n;
        jobs[t].out = out + lo;
        jobs[t].n = hi - lo;
        jobs[t].seed = seed;
        jobs[t].offset = offset + lo;
        joined[t] = pthread_create(&th[t], NULL, fill_thread, &jobs[t]) == 0;
        if (!joined[t]) fill_thread(&jobs[t]); /* no thread: do the range here */
        used = t + 1;
    }
    for (int t = 0; t < used; t++)
        if (joined[t]) pthread_join(th[t], NULL);
    return 0;
}
