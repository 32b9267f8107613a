// Saving and loading deflation data (the one-off, expensive part of the
// method: Sec. 5 amortises the critical eigenvectors over many evaluations;
// a file lets later processes reuse them).
//
// File layout (little-endian, as the host writes it):
//   char[8]  "OVLDEFL1"
//   int32    dims[4], antiperiodic_t, scheme, m, setup_restarts, setup_matvecs, 0
//   double   mu, m_w
//   uint64   link fingerprint (ovl_set_links), N = 12 V
//   double   T (Schur: m x m column-major complex) or Lambda (LR: m complex)
//   double   S or R: m canonical complex128 spinors
//   double   L: m canonical spinors (LR only)
//   uint64   FNV-1a 64 of every byte before it
// Loading checks the magic, the operator (dims, boundary, link fingerprint),
// the sizes and the checksum; the caller's mu and m_w are recorded in the
// object as in ovl_set_deflation, so a solve with other values is rejected.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "ovl_common.cuh"

namespace {

struct Header {
    char magic[8];
    int32_t dims[4], apbc, scheme, m, restarts, matvecs, pad;
    double mu, m_w;
    uint64_t link_hash, N;
};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* c = (const unsigned char*)p;
        for (size_t i = 0; i < n; i++) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
};

struct File {
    FILE* f;
    explicit File(FILE* g) : f(g) {}
    ~File() {
        if (f) fclose(f);
    }
};

}  // namespace

extern "C" int ovl_deflation_save(ovl_deflation d, const char* path) {
    if (!d || !path) return ovl_fail(d ? d->lat : nullptr, OVL_EINVAL, "ovl_deflation_save: null argument");
    ovl_lattice lat = d->lat;
    const size_t N = lat->N, m = (size_t)d->m;
    Header h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "OVLDEFL1", 8);
    for (int i = 0; i < 4; i++) h.dims[i] = lat->dims[i];
    h.apbc = lat->apbc;
    h.scheme = d->scheme;
    h.m = d->m;
    h.restarts = d->setup_restarts;
    h.matvecs = d->setup_matvecs;
    h.mu = d->mu;
    h.m_w = d->m_w;
    h.link_hash = lat->link_hash;
    h.N = N;
    std::vector<double> S(2 * N * m), L(d->scheme == OVL_DEFL_LR ? 2 * N * m : 0);
    if (int rc = ovl_get_deflation(d, nullptr, nullptr, S.data(), nullptr, L.empty() ? nullptr : L.data())) return rc;
    File f(fopen(path, "wb"));
    if (!f.f) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_save: cannot open %s for writing", path);
    Fnv sum;
    auto put = [&](const void* p, size_t n) -> bool {
        sum.add(p, n);
        return fwrite(p, 1, n, f.f) == n;
    };
    bool ok = put(&h, sizeof h) && put(d->T_host.data(), d->T_host.size() * sizeof(double)) &&
              put(S.data(), S.size() * sizeof(double)) && (L.empty() || put(L.data(), L.size() * sizeof(double)));
    uint64_t c = sum.h;
    ok = ok && fwrite(&c, 1, sizeof c, f.f) == sizeof c;
    if (!ok) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_save: writing %s failed", path);
    return OVL_OK;
}

extern "C" int ovl_deflation_load(ovl_lattice lat, const char* path, ovl_deflation* out) {
    if (!lat || !path || !out) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: null argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: links not set");
    File f(fopen(path, "rb"));
    if (!f.f) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: cannot open %s", path);
    Header h;
    Fnv sum;
    auto get = [&](void* p, size_t n) -> bool {
        if (fread(p, 1, n, f.f) != n) return false;
        sum.add(p, n);
        return true;
    };
    if (!get(&h, sizeof h) || memcmp(h.magic, "OVLDEFL1", 8) != 0)
        return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: %s is not a deflation file", path);
    for (int i = 0; i < 4; i++)
        if (h.dims[i] != lat->dims[i])
            return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: lattice %dx%dx%dx%d in the file, %dx%dx%dx%d here",
                            h.dims[0], h.dims[1], h.dims[2], h.dims[3], lat->dims[0], lat->dims[1], lat->dims[2],
                            lat->dims[3]);
    if (h.apbc != lat->apbc || h.N != lat->N)
        return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: boundary condition or size differs");
    if (h.link_hash != lat->link_hash)
        return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: the file belongs to other links (fingerprint %016llx, "
                        "lattice %016llx)", (unsigned long long)h.link_hash, (unsigned long long)lat->link_hash);
    if ((h.scheme != OVL_DEFL_SCHUR && h.scheme != OVL_DEFL_LR) || h.m < 1 || h.m > 200)
        return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: bad scheme %d or m %d", h.scheme, h.m);
    const size_t N = lat->N, m = (size_t)h.m;
    std::vector<double> T(h.scheme == OVL_DEFL_SCHUR ? 2 * m * m : 2 * m), S(2 * N * m),
        L(h.scheme == OVL_DEFL_LR ? 2 * N * m : 0);
    uint64_t c = 0;
    bool ok = get(T.data(), T.size() * sizeof(double)) && get(S.data(), S.size() * sizeof(double)) &&
              (L.empty() || get(L.data(), L.size() * sizeof(double)));
    const uint64_t expect = sum.h;
    ok = ok && fread(&c, 1, sizeof c, f.f) == sizeof c && c == expect;
    if (!ok) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_load: %s is truncated or damaged", path);
    ovl_deflation d = nullptr;
    if (int rc = ovl_set_deflation(lat, h.mu, h.m_w, h.scheme, h.m, S.data(), T.data(), L.empty() ? nullptr : L.data(),
                                   &d))
        return rc;
    d->setup_restarts = h.restarts;
    d->setup_matvecs = h.matvecs;
    *out = d;
    return OVL_OK;
}
