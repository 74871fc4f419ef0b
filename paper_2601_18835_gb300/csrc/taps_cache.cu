// Tap banks on disk: rfd_taps_key (a SHA-256 digest of every input that decides rfd_make_taps'
// outputs) and rfd_make_taps_cached (load the bank named by that digest, else compute and
// store it).  Tap extraction (Sec. V) is the set-up's dominant cost and depends only on the
// grid, the PSD, the bank and the tap policy, so a later run on the same bank reads it back.
//
// SHA-256 follows FIPS 180-4.  Its round constants are the first 32 fractional bits of the cube
// roots of the first 64 primes and its initial hash the same of the square roots of the first 8;
// both are computed here by exact integer roots rather than tabulated.
//
// File <cache_dir>/<64 hex digits of the key>.rfdtaps: the 8-byte magic "RFDTAPS" 0x01, a
// little-endian uint64 header length, a JSON header (key, n_tmpl, k_stride, has_match and the
// sections with dtype, shape, offset, bytes), then the sections, each 64-byte aligned from the
// end of the header: taps complex64 [n_tmpl][k_stride], K int32 [n_tmpl], lag int32 [n_tmpl],
// sigma_eff float64 [n_tmpl] and, when has_match, match float64 [n_tmpl].
#include "internal.cuh"

#include <nvtx3/nvToolsExt.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstring>
#include <string>

namespace rfd {
namespace {

// ------------------------------------------------------------------ SHA-256 (FIPS 180-4)
struct Sha256Tables {
    uint32_t k[64];
    uint32_t h0[8];
};

// floor(x) for x = root-th root of v (v < 2^110), exactly, from a floating-point first guess.
uint64_t int_root(unsigned __int128 v, int root) {
    auto pw = [root](unsigned __int128 x) { return root == 2 ? x * x : x * x * x; };
    uint64_t x = (uint64_t)(root == 2 ? std::sqrt((double)v) : std::cbrt((double)v));
    while (x > 0 && pw(x) > v) --x;
    while (pw((unsigned __int128)x + 1) <= v) ++x;
    return x;
}

const Sha256Tables &sha256_tables() {
    static const Sha256Tables t = [] {
        Sha256Tables s{};
        int primes[64], np = 0;
        for (int c = 2; np < 64; ++c) {
            bool prime = true;
            for (int d = 2; d * d <= c; ++d) prime = prime && (c % d != 0);
            if (prime) primes[np++] = c;
        }
        for (int i = 0; i < 64; ++i)     // cbrt(p) 2^32 = cbrt(p 2^96): keep its low 32 bits
            s.k[i] = (uint32_t)int_root((unsigned __int128)primes[i] << 96, 3);
        for (int i = 0; i < 8; ++i)      // sqrt(p) 2^32 = sqrt(p 2^64)
            s.h0[i] = (uint32_t)int_root((unsigned __int128)primes[i] << 64, 2);
        return s;
    }();
    return t;
}

class Sha256 {
public:
    Sha256() {
        const Sha256Tables &t = sha256_tables();
        std::memcpy(h_, t.h0, sizeof h_);
    }
    void update(const void *data, size_t n) {
        const uint8_t *p = (const uint8_t *)data;
        total_ += n;
        while (n > 0) {
            const size_t take = std::min(n, (size_t)64 - fill_);
            std::memcpy(buf_ + fill_, p, take);
            fill_ += take;
            p += take;
            n -= take;
            if (fill_ == 64) {
                block(buf_);
                fill_ = 0;
            }
        }
    }
    void finish(uint8_t out[32]) {
        const uint64_t bits = total_ * 8;
        const uint8_t one = 0x80, zero = 0;
        update(&one, 1);
        while (fill_ != 56) update(&zero, 1);
        uint8_t len[8];
        for (int i = 0; i < 8; ++i) len[i] = (uint8_t)(bits >> (56 - 8 * i));
        update(len, 8);
        for (int i = 0; i < 8; ++i)
            for (int b = 0; b < 4; ++b) out[4 * i + b] = (uint8_t)(h_[i] >> (24 - 8 * b));
    }

private:
    static uint32_t rotr(uint32_t x, int r) { return (x >> r) | (x << (32 - r)); }
    void block(const uint8_t *m) {
        const uint32_t *k = sha256_tables().k;
        uint32_t w[64];
        for (int t = 0; t < 16; ++t)
            w[t] = (uint32_t)m[4 * t] << 24 | (uint32_t)m[4 * t + 1] << 16 | (uint32_t)m[4 * t + 2] << 8 |
                   (uint32_t)m[4 * t + 3];
        for (int t = 16; t < 64; ++t) {
            const uint32_t s0 = rotr(w[t - 15], 7) ^ rotr(w[t - 15], 18) ^ (w[t - 15] >> 3);
            const uint32_t s1 = rotr(w[t - 2], 17) ^ rotr(w[t - 2], 19) ^ (w[t - 2] >> 10);
            w[t] = w[t - 16] + s0 + w[t - 7] + s1;
        }
        uint32_t a = h_[0], b = h_[1], c = h_[2], d = h_[3], e = h_[4], f = h_[5], g = h_[6], h = h_[7];
        for (int t = 0; t < 64; ++t) {
            const uint32_t t1 = h + (rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25)) + ((e & f) ^ (~e & g)) + k[t] + w[t];
            const uint32_t t2 = (rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22)) + ((a & b) ^ (a & c) ^ (b & c));
            h = g;
            g = f;
            f = e;
            e = d + t1;
            d = c;
            c = b;
            b = a;
            a = t1 + t2;
        }
        h_[0] += a;
        h_[1] += b;
        h_[2] += c;
        h_[3] += d;
        h_[4] += e;
        h_[5] += f;
        h_[6] += g;
        h_[7] += h;
    }
    uint32_t h_[8];
    uint8_t buf_[64];
    size_t fill_ = 0;
    uint64_t total_ = 0;
};

bool little_endian() {
    const uint16_t x = 1;
    uint8_t b;
    std::memcpy(&b, &x, 1);
    return b == 1;
}

template <typename T>
void put(Sha256 &h, T v) {
    h.update(&v, sizeof v);
}

// ------------------------------------------------------------------ the file
constexpr char kMagic[8] = {'R', 'F', 'D', 'T', 'A', 'P', 'S', 1};

size_t align64(size_t x) { return (x + 63) / 64 * 64; }

struct Section {
    const char *name, *dtype;
    int64_t rows, cols;
    size_t bytes;
};

std::vector<Section> sections(int32_t n_tmpl, int32_t k_stride, bool has_match) {
    const size_t n = (size_t)n_tmpl;
    std::vector<Section> s = {{"taps", "c64", n_tmpl, k_stride, n * (size_t)k_stride * 8},
                              {"k", "i32", n_tmpl, 1, n * 4},
                              {"lag", "i32", n_tmpl, 1, n * 4},
                              {"sigma_eff", "f64", n_tmpl, 1, n * 8}};
    if (has_match) s.push_back({"match", "f64", n_tmpl, 1, n * 8});
    return s;
}

bool header_number(const std::string &h, const char *key, double *out) {
    const std::string k = std::string("\"") + key + "\": ";
    const size_t at = h.find(k);
    if (at == std::string::npos) return false;
    char *end = nullptr;
    *out = std::strtod(h.c_str() + at + k.size(), &end);
    return end != h.c_str() + at + k.size();
}

std::string hex(const uint8_t key[32]) {
    static const char d[] = "0123456789abcdef";
    std::string s(64, '0');
    for (int i = 0; i < 32; ++i) {
        s[2 * i] = d[key[i] >> 4];
        s[2 * i + 1] = d[key[i] & 15];
    }
    return s;
}

// The host image of one tap bank.
struct Bank {
    std::vector<char> taps;
    std::vector<int32_t> k, lag;
    std::vector<double> sigma, match;
};

// Reads `path` when it holds this key, n_tmpl and k_stride (and a match section when
// want_match) with sane contents; false on any mismatch, truncation or missing file.
bool read_bank(const std::string &path, const std::string &key_hex, int32_t n_tmpl, int32_t k_stride, int64_t n,
               bool want_match, Bank *b) {
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return false;
    char magic[8];
    uint64_t hl = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&hl, 8, 1, f) == 1 && hl > 0 && hl < (1u << 20);
    std::string h;
    if (ok) {
        h.resize(hl);
        ok = std::fread(&h[0], 1, hl, f) == hl;
    }
    double v_n = -1, v_s = -1, v_m = -1;
    ok = ok && h.find("\"key\": \"" + key_hex + "\"") != std::string::npos && header_number(h, "n_tmpl", &v_n) &&
         header_number(h, "k_stride", &v_s) && header_number(h, "has_match", &v_m) && (int64_t)v_n == n_tmpl &&
         (int64_t)v_s == k_stride && (v_m == 0 || v_m == 1) && (!want_match || v_m == 1);
    if (ok) {
        const std::vector<Section> secs = sections(n_tmpl, k_stride, v_m == 1);
        b->taps.resize(secs[0].bytes);
        b->k.resize(n_tmpl);
        b->lag.resize(n_tmpl);
        b->sigma.resize(n_tmpl);
        b->match.resize(v_m == 1 ? n_tmpl : 0);
        void *dst[5] = {b->taps.data(), b->k.data(), b->lag.data(), b->sigma.data(), b->match.data()};
        size_t off = 0;
        for (size_t i = 0; ok && i < secs.size(); ++i) {
            ok = secs[i].bytes == 0 || std::fread(dst[i], 1, secs[i].bytes, f) == secs[i].bytes;
            const size_t pad = align64(off + secs[i].bytes) - (off + secs[i].bytes);
            char skip[64];
            ok = ok && (pad == 0 || std::fread(skip, 1, pad, f) == pad);
            off = align64(off + secs[i].bytes);
        }
        ok = ok && std::fgetc(f) == EOF;
    }
    std::fclose(f);
    for (int32_t j = 0; ok && j < n_tmpl; ++j)
        ok = b->k[j] >= 1 && b->k[j] <= k_stride && b->lag[j] >= -(n / 2) && b->lag[j] < n / 2 &&
             std::isfinite(b->sigma[j]) && b->sigma[j] >= 0;
    return ok;
}

rfd_status write_bank(const std::string &path, const std::string &key_hex, int32_t n_tmpl, int32_t k_stride,
                      const Bank &b) {
    const bool has_match = !b.match.empty();
    const std::vector<Section> secs = sections(n_tmpl, k_stride, has_match);
    char buf[256];
    std::snprintf(buf, sizeof buf, "{\"format\": \"librfd tap bank\", \"version\": 1, \"key\": \"%s\", "
                  "\"n_tmpl\": %d, \"k_stride\": %d, \"has_match\": %d, \"sections\": [", key_hex.c_str(), n_tmpl,
                  k_stride, has_match ? 1 : 0);
    std::string h = buf;
    size_t off = 0;
    for (size_t i = 0; i < secs.size(); ++i) {
        std::snprintf(buf, sizeof buf, "%s{\"name\": \"%s\", \"dtype\": \"%s\", \"shape\": [%lld, %lld], "
                      "\"offset\": %zu, \"bytes\": %zu}", i ? ", " : "", secs[i].name, secs[i].dtype,
                      (long long)secs[i].rows, (long long)secs[i].cols, off, secs[i].bytes);
        h += buf;
        off = align64(off + secs[i].bytes);
    }
    h += "]}\n";
    // a temporary name in the same directory, then rename: a reader never sees a partial file
    const std::string tmp = path + ".tmp." + std::to_string((long long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "wb");
    RFD_REQUIRE(f, RFD_ERR_ARG, "make_taps_cached: cannot write %s (%s)", tmp.c_str(), std::strerror(errno));
    const uint64_t hl = h.size();
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&hl, 8, 1, f) == 1 &&
              std::fwrite(h.data(), 1, h.size(), f) == h.size();
    const void *src[5] = {b.taps.data(), b.k.data(), b.lag.data(), b.sigma.data(), b.match.data()};
    const char zeros[64] = {0};
    off = 0;
    for (size_t i = 0; ok && i < secs.size(); ++i) {
        ok = secs[i].bytes == 0 || std::fwrite(src[i], 1, secs[i].bytes, f) == secs[i].bytes;
        const size_t pad = align64(off + secs[i].bytes) - (off + secs[i].bytes);
        ok = ok && (pad == 0 || std::fwrite(zeros, 1, pad, f) == pad);
        off = align64(off + secs[i].bytes);
    }
    ok = (std::fclose(f) == 0) && ok;
    if (ok) ok = std::rename(tmp.c_str(), path.c_str()) == 0;
    if (!ok) std::remove(tmp.c_str());
    RFD_REQUIRE(ok, RFD_ERR_ARG, "make_taps_cached: writing %s failed (%s)", path.c_str(), std::strerror(errno));
    return RFD_OK;
}

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace
}  // namespace rfd

extern "C" {

rfd_status rfd_taps_key(const rfd_grid *grid, const double *psd_host, const rfd_params *refs_host, int32_t n_ref,
                        const rfd_params *tmpl_host, const int32_t *ref_of_tmpl_host, int32_t n_tmpl,
                        const int32_t *k_host, const int32_t *buckets_host, int32_t n_buckets, double energy_frac,
                        int32_t k_stride, double tukey_alpha, uint8_t *key_out) {
    using namespace rfd;
    RFD_REQUIRE(little_endian(), RFD_ERR_UNSUPPORTED, "taps_key: the serialisation is defined for little-endian hosts");
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 1 && n_tmpl >= 0, RFD_ERR_SHAPE, "need n_ref >= 1 and n_tmpl >= 0");
    RFD_REQUIRE(psd_host && refs_host && key_out && (n_tmpl == 0 || (tmpl_host && ref_of_tmpl_host)), RFD_ERR_ARG,
                "NULL argument");
    RFD_REQUIRE(k_host || n_tmpl == 0 || (buckets_host && n_buckets >= 1), RFD_ERR_ARG,
                "give either k_host or a non-empty bucket list");
    const int32_t mode = k_host ? 0 : 1;
    Sha256 h;
    h.update("librfd-taps", 12);                 // the 11 characters and their terminating NUL
    put<int32_t>(h, RFD_VERSION);
    put<int32_t>(h, mode);
    put<double>(h, grid->fs);
    put<int64_t>(h, grid->n);
    put<double>(h, grid->f_low);
    put<int32_t>(h, grid->pn_flags);
    put<int32_t>(h, n_ref);
    put<int32_t>(h, n_tmpl);
    put<int32_t>(h, k_stride);
    put<double>(h, tukey_alpha);
    put<double>(h, mode ? energy_frac : 0.0);
    put<int32_t>(h, mode ? n_buckets : 0);
    h.update(refs_host, sizeof(rfd_params) * (size_t)n_ref);
    h.update(tmpl_host, sizeof(rfd_params) * (size_t)n_tmpl);
    h.update(ref_of_tmpl_host, sizeof(int32_t) * (size_t)n_tmpl);
    if (mode == 0)
        h.update(k_host, sizeof(int32_t) * (size_t)n_tmpl);
    else
        h.update(buckets_host, sizeof(int32_t) * (size_t)n_buckets);
    h.update(psd_host, sizeof(double) * (size_t)g.nf);
    h.finish(key_out);
    return RFD_OK;
}

rfd_status rfd_make_taps_cached(const char *cache_dir, rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                                const rfd_params *refs_host, int32_t n_ref, const rfd_params *tmpl_host,
                                const int32_t *ref_of_tmpl_host, int32_t n_tmpl, const int32_t *k_host,
                                const int32_t *buckets_host, int32_t n_buckets, double energy_frac, int32_t k_stride,
                                double tukey_alpha, void *taps_dev, int32_t *k_dev, int32_t *lag_dev,
                                double *sigma_dev, double *match_dev, int32_t *hit_host, void *stream) {
    using namespace rfd;
    NvtxRange nvtx_range("rfd_make_taps_cached");
    RFD_REQUIRE(cache_dir && *cache_dir && hit_host && ctx && psd_dev, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(n_tmpl >= 1, RFD_ERR_SHAPE, "make_taps_cached: n_tmpl must be >= 1");
    RFD_REQUIRE(taps_dev && lag_dev && sigma_dev, RFD_ERR_ARG, "NULL output");
    RFD_REQUIRE(k_stride >= 1 && k_stride <= 4096, RFD_ERR_SHAPE, "k_stride=%d must be in [1, 4096]", k_stride);
    *hit_host = 0;
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> psd((size_t)g.nf);
    RFD_TRY_CUDA(cudaMemcpyAsync(psd.data(), psd_dev, psd.size() * 8, cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    uint8_t key[32];
    RFD_TRY(rfd_taps_key(grid, psd.data(), refs_host, n_ref, tmpl_host, ref_of_tmpl_host, n_tmpl, k_host,
                         buckets_host, n_buckets, energy_frac, k_stride, tukey_alpha, key));
    const std::string key_hex = hex(key);
    const std::string path = std::string(cache_dir) + "/" + key_hex + ".rfdtaps";
    const size_t J = (size_t)n_tmpl;
    Bank b;
    if (read_bank(path, key_hex, n_tmpl, k_stride, g.n, match_dev != nullptr, &b)) {
        RFD_TRY_CUDA(cudaMemcpyAsync(taps_dev, b.taps.data(), b.taps.size(), cudaMemcpyHostToDevice, s));
        RFD_TRY_CUDA(cudaMemcpyAsync(lag_dev, b.lag.data(), J * 4, cudaMemcpyHostToDevice, s));
        RFD_TRY_CUDA(cudaMemcpyAsync(sigma_dev, b.sigma.data(), J * 8, cudaMemcpyHostToDevice, s));
        if (k_dev) RFD_TRY_CUDA(cudaMemcpyAsync(k_dev, b.k.data(), J * 4, cudaMemcpyHostToDevice, s));
        if (match_dev) RFD_TRY_CUDA(cudaMemcpyAsync(match_dev, b.match.data(), J * 8, cudaMemcpyHostToDevice, s));
        RFD_TRY_CUDA(cudaStreamSynchronize(s));
        *hit_host = 1;
        return RFD_OK;
    }
    // a miss: extract the taps, then store them under the key
    int32_t *k_out = k_dev;
    void *k_tmp = nullptr;
    if (!k_out && !k_host) {
        RFD_TRY_CUDA(cudaMalloc(&k_tmp, J * 4));
        k_out = (int32_t *)k_tmp;
    }
    rfd_status st = rfd_make_taps(ctx, grid, psd_dev, refs_host, n_ref, tmpl_host, ref_of_tmpl_host, n_tmpl, k_host,
                                  buckets_host, n_buckets, energy_frac, k_stride, tukey_alpha, taps_dev, k_out,
                                  lag_dev, sigma_dev, match_dev, stream);
    if (st == RFD_OK) {
        b.taps.resize(J * (size_t)k_stride * 8);
        b.k.resize(J);
        b.lag.resize(J);
        b.sigma.resize(J);
        b.match.resize(match_dev ? J : 0);
        cudaError_t e = cudaMemcpyAsync(b.taps.data(), taps_dev, b.taps.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.lag.data(), lag_dev, J * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.sigma.data(), sigma_dev, J * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && k_out) e = cudaMemcpyAsync(b.k.data(), k_out, J * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && match_dev)
            e = cudaMemcpyAsync(b.match.data(), match_dev, J * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("make_taps_cached: reading the taps back failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
        }
        if (st == RFD_OK && !k_out) std::memcpy(b.k.data(), k_host, J * 4);
    }
    if (k_tmp) cudaFree(k_tmp);
    RFD_TRY(st);
    if (::mkdir(cache_dir, 0755) != 0 && errno != EEXIST) {
        set_error("make_taps_cached: cannot create %s (%s); the outputs hold the extracted taps", cache_dir,
                  std::strerror(errno));
        return RFD_ERR_ARG;
    }
    return write_bank(path, key_hex, n_tmpl, k_stride, b);
}

}  // extern "C"
