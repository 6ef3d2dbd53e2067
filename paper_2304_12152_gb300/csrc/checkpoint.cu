// Policy checkpoints: host-only save / load of a policy's descriptor, canonical
// float32 weights and biases, FP8 activation scales and the training iteration, so
// that a training run (Algorithm 1, TRAIN step, repeated for many iterations) can
// stop and resume.  No device memory, stream or CUDA call is involved.
//
// File layout, little-endian:
//   "HTCKPT01"                       8-byte tag
//   u32 header_bytes                 length of the header that follows
//   header: i32 n_layers, i32 channels[n_layers + 1], i32 head, i32 precision,
//           i32 levels, i32 arch, i64 step, f32 act_scale[n_layers],
//           i64 n_weights, i64 n_biases
//   f32 weights[n_weights]           OIHW per layer, layers concatenated
//   f32 biases[n_biases]
//   u64 checksum                     FNV-1a (64-bit) of every byte before it
// A file is written to "<path>.tmp" and renamed over <path>, so an interrupted save
// leaves any earlier checkpoint intact.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "ht_internal.cuh"

namespace {

constexpr char kTag[8] = {'H', 'T', 'C', 'K', 'P', 'T', '0', '1'};

struct Writer {
    std::vector<unsigned char> b;
    void u32(uint32_t v)
    {
        for (int i = 0; i < 4; ++i) b.push_back((unsigned char)(v >> (8 * i)));
    }
    void u64(uint64_t v)
    {
        for (int i = 0; i < 8; ++i) b.push_back((unsigned char)(v >> (8 * i)));
    }
    void i32(int32_t v) { u32((uint32_t)v); }
    void i64(int64_t v) { u64((uint64_t)v); }
    void f32(float v)
    {
        uint32_t u;
        memcpy(&u, &v, 4);
        u32(u);
    }
};

struct Reader {
    const unsigned char *p;
    size_t n, at = 0;
    bool ok = true;
    uint64_t get(int bytes)
    {
        if (!ok || n - at < (size_t)bytes) {
            ok = false;
            return 0;
        }
        uint64_t v = 0;
        for (int i = 0; i < bytes; ++i) v |= (uint64_t)p[at + i] << (8 * i);
        at += (size_t)bytes;
        return v;
    }
    int32_t i32() { return (int32_t)(uint32_t)get(4); }
    int64_t i64() { return (int64_t)get(8); }
    float f32()
    {
        const uint32_t u = (uint32_t)get(4);
        float v;
        memcpy(&v, &u, 4);
        return v;
    }
};

uint64_t fnv1a64(const unsigned char *p, size_t n)
{
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

void param_counts(const ht_policy_desc *d, int64_t *nw, int64_t *nb)
{
    *nw = *nb = 0;
    for (int l = 0; l < d->n_layers; ++l) {
        *nw += (int64_t)d->channels[l + 1] * d->channels[l] * 9;
        *nb += d->channels[l + 1];
    }
}

ht_status io_error(const char *what, const char *path)
{
    ht_set_error("checkpoint %s: %s", path, what);
    return HT_ERR_IO;
}

// Parses a whole file image; fills info and, when w / b are given, the arrays.
ht_status parse(const std::vector<unsigned char> &img, const char *path, ht_checkpoint_info *info, float *w,
                int64_t w_cap, float *b, int64_t b_cap)
{
    if (img.size() < sizeof(kTag) + 4 + 8 || memcmp(img.data(), kTag, sizeof(kTag)) != 0)
        return io_error("not a policy checkpoint (bad tag or too short)", path);
    const size_t body = img.size() - 8;
    Reader tail{img.data() + body, 8};
    if (tail.get(8) != fnv1a64(img.data(), body)) return io_error("checksum mismatch (corrupt file)", path);

    Reader r{img.data(), body};
    r.at = sizeof(kTag);
    const uint32_t header_bytes = (uint32_t)r.get(4);
    const size_t header_end = r.at + header_bytes;
    ht_checkpoint_info ci;
    memset(&ci, 0, sizeof(ci));
    ci.desc.n_layers = r.i32();
    if (!r.ok || ci.desc.n_layers < 1 || ci.desc.n_layers > HT_MAX_LAYERS)
        return io_error("layer count out of range", path);
    for (int l = 0; l <= ci.desc.n_layers; ++l) ci.desc.channels[l] = r.i32();
    ci.desc.head = r.i32();
    ci.desc.precision = r.i32();
    ci.desc.levels = r.i32();
    ci.desc.arch = r.i32();
    ci.step = r.i64();
    for (int l = 0; l < ci.desc.n_layers; ++l) ci.act_scale[l] = r.f32();
    ci.n_weights = r.i64();
    ci.n_biases = r.i64();
    if (!r.ok || r.at != header_end) return io_error("malformed header", path);
    if (ht_validate_desc(&ci.desc) != HT_OK) return io_error("header holds an invalid policy descriptor", path);
    int64_t nw, nb;
    param_counts(&ci.desc, &nw, &nb);
    if (ci.n_weights != nw || ci.n_biases != nb) return io_error("parameter counts do not match the layers", path);
    if ((uint64_t)(body - r.at) != (uint64_t)(nw + nb) * 4u) return io_error("truncated or oversized parameter block", path);
    if (w || b) {
        HT_CHECK_ARG(w && b, "weights and biases are read together");
        HT_CHECK_ARG(w_cap >= nw && b_cap >= nb, "output arrays too small: need %lld weights and %lld biases",
                     (long long)nw, (long long)nb);
        for (int64_t i = 0; i < nw; ++i) w[i] = r.f32();
        for (int64_t i = 0; i < nb; ++i) b[i] = r.f32();
    }
    *info = ci;
    return HT_OK;
}

}  // namespace

extern "C" ht_status ht_checkpoint_save(const char *path, const ht_policy_desc *desc, const float *weights_host,
                                        const float *biases_host, const float *act_scales_host, int64_t step)
{
    HT_RANGE("ht_checkpoint_save");
    HT_CHECK_ARG(path && path[0], "empty checkpoint path");
    HT_CHECK_ARG(weights_host && biases_host, "weights and biases are required");
    HT_CHECK_ARG(step >= 0, "negative step");
    const ht_status st = ht_validate_desc(desc);
    if (st != HT_OK) return st;
    int64_t nw, nb;
    param_counts(desc, &nw, &nb);

    Writer hd;
    hd.i32(desc->n_layers);
    for (int l = 0; l <= desc->n_layers; ++l) hd.i32(desc->channels[l]);
    hd.i32(desc->head);
    hd.i32(desc->precision);
    hd.i32(desc->levels);
    hd.i32(desc->arch);
    hd.i64(step);
    for (int l = 0; l < desc->n_layers; ++l) hd.f32(act_scales_host ? act_scales_host[l] : 1.f);
    hd.i64(nw);
    hd.i64(nb);

    Writer f;
    f.b.reserve(sizeof(kTag) + 4 + hd.b.size() + (size_t)(nw + nb) * 4 + 8);
    f.b.insert(f.b.end(), kTag, kTag + sizeof(kTag));
    f.u32((uint32_t)hd.b.size());
    f.b.insert(f.b.end(), hd.b.begin(), hd.b.end());
    for (int64_t i = 0; i < nw; ++i) f.f32(weights_host[i]);
    for (int64_t i = 0; i < nb; ++i) f.f32(biases_host[i]);
    f.u64(fnv1a64(f.b.data(), f.b.size()));

    std::vector<char> tmp(strlen(path) + 5);
    snprintf(tmp.data(), tmp.size(), "%s.tmp", path);
    FILE *fp = fopen(tmp.data(), "wb");
    if (!fp) return io_error("cannot open for writing", tmp.data());
    const bool wrote = fwrite(f.b.data(), 1, f.b.size(), fp) == f.b.size();
    const bool closed = fclose(fp) == 0;
    if (!wrote || !closed) {
        remove(tmp.data());
        return io_error("write failed", tmp.data());
    }
    if (rename(tmp.data(), path) != 0) {
        remove(tmp.data());
        return io_error("cannot replace the file", path);
    }
    return HT_OK;
}

extern "C" ht_status ht_checkpoint_load(const char *path, ht_checkpoint_info *info, float *weights_host,
                                        int64_t weights_cap, float *biases_host, int64_t biases_cap)
{
    HT_RANGE("ht_checkpoint_load");
    HT_CHECK_ARG(path && path[0], "empty checkpoint path");
    HT_CHECK_ARG(info != nullptr, "null info pointer");
    FILE *fp = fopen(path, "rb");
    if (!fp) return io_error("cannot open for reading", path);
    std::vector<unsigned char> img;
    unsigned char buf[1 << 16];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), fp)) > 0) img.insert(img.end(), buf, buf + got);
    const bool err = ferror(fp) != 0;
    fclose(fp);
    if (err) return io_error("read failed", path);
    return parse(img, path, info, weights_host, weights_cap, biases_host, biases_cap);
}
