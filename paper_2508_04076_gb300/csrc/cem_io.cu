// Checkpoint and resume: the dynamic state of a context to a file and back.
//
// A checkpoint holds everything a step reads that is not fixed by the mesh
// description and the material: node, element and edge arrays up to their
// current counts, the fan and incidence pools up to their tops, the crack
// records of the input elements, the candidate list, the new-node and
// new-edge maps, U_d, the counters, and the node storage order with the node
// references a renumbering rewrites.  The step's scratch (element strains,
// edge stresses, element forces, flags) is rewritten before it is read and is
// not saved.  A context built from the same description and material and then
// loaded continues bit for bit as the saved one would have.
//
// File layout (host byte order): the 8-byte tag "CEMCKPT3", a header of int64
// fields (HDR_* below), then every array as raw bytes in a fixed order, each
// preceded by its byte count, and last a 64-bit FNV-1a hash of every byte
// before it.  Loading reads and hashes the whole file before it changes the
// context, so a truncated or corrupted file leaves the context as it was
// Every index array is also range-checked on the host in that first pass
// (node, element, edge and pool indices, the storage order a permutation,
// every list inside its pool's used part), so a file that cem_save did not
// write cannot put an out-of-range index on the device.
#include "cem_common.cuh"

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

enum {
    HDR_ELEM, HDR_PREC, HDR_N0, HDR_T0, HDR_E0, HDR_NC, HDR_TC, HDR_EC, HDR_FANCAP, HDR_INCCAP, HDR_HASHCAP,
    HDR_NINST, HDR_SPLITMODE, HDR_N, HDR_T, HDR_E, HDR_NCAND, HDR_NSPLITALL, HDR_NSPLITRUN, HDR_NACTIVE,
    HDR_FANTOP, HDR_INCTOP, HDR_STEP, HDR_DT_BITS, HDR_RENUMBERED, HDR_REORDER_N, HDR_NREORDER, HDR_COUNT
};
const char TAG[8] = {'C', 'E', 'M', 'C', 'K', 'P', 'T', '3'};

// 64-bit FNV-1a (Fowler, Noll, Vo): offset basis and prime as published.
const uint64_t FNV_BASIS = 0xcbf29ce484222325ull, FNV_PRIME = 0x100000001b3ull;
uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * FNV_PRIME;
    return h;
}

// One array slice: device pointer, bytes; for int32 index arrays the range
// [lo, hi) every entry must lie in (hi = 0: not an index array), with -1 also
// allowed where `unset` says so.
struct Field {
    void* p;
    size_t bytes;
    int64_t lo = 0, hi = 0;
    bool unset = false;
};

// The saved arrays, in file order (null pointers are skipped consistently on both sides).
std::vector<Field> fields(cem_ctx* c) {
    std::vector<Field> f;
    auto add = [&](void* p, int64_t n, size_t esz) {
        if (p && n > 0) f.push_back({p, (size_t)n * esz});
    };
    // an int32 index array with entries in [lo, hi) (or -1 if unset)
    auto idx = [&](void* p, int64_t n, int64_t lo, int64_t hi, bool unset = false) {
        if (p && n > 0) f.push_back({p, (size_t)n * 4, lo, hi, unset});
    };
    auto rows = [&](void* p, int nrow, int64_t ld, int64_t n, size_t esz) {
        for (int r = 0; r < nrow && p; ++r) add((char*)p + (size_t)r * ld * esz, n, esz);
    };
    auto idx_rows = [&](int* p, int nrow, int64_t ld, int64_t n, int64_t lo, int64_t hi) {
        for (int r = 0; r < nrow && p; ++r) idx(p + (size_t)r * ld, n, lo, hi);
    };
    const int64_t N = c->N, T = c->T, E = c->E;
    const bool hex = c->elem_type == CEM_ELEM_HEX8;
    rows(c->X, 3, c->Nc, N, 8);
    rows(c->u, 3, c->Nc, N, 8);
    rows(c->v, 3, c->Nc, N, 8);
    rows(c->a, 3, c->Nc, N, 8);
    rows(c->fext, 3, c->Nc, N, 8);
    add(c->mass, N, 8);
    add(c->minv, N, 8);
    idx(c->inc_off, N, 0, std::max<int64_t>(c->inc_top, 1));
    idx(c->inc_cnt, N, 0, c->inc_top + 1);
    add(c->dtn, N, 8);
    add(c->node_inst, N, 4);
    add(c->uhl, 8 * N, 4);
    idx_rows(c->conn, c->npe, c->Tc, T, 0, N);
    idx_rows(c->t2e, c->epe, c->Tc, T, 0, E);
    idx(c->anc, T, 0, c->T0);
    add(c->active, T, 1);
    const int ng = hex ? (int)cem_hex_geometry_values() : 9;
    rows(c->Vg, ng, c->Tc, T, 8);
    rows(c->Vg32, ng, c->Tc, T, 4);
    add(c->vol, T, 8);
    add(c->lam, T, 8);
    add(c->mu, T, 8);
    idx(c->fan_off, E, 0, std::max<int64_t>(c->fan_top, 1));
    idx(c->fan_cnt, E, 0, c->fan_top + 1);
    add(c->cl, E, 8);
    add(c->cm, E, 8);
    add(c->sumV, E, 8);
    add(c->cl32, E, 4);
    add(c->cm32, E, 4);
    idx(c->fan_pool, c->fan_top, 0, hex ? T * c->epe : T);   // fan entries: elements (hexahedra: element * 12 + edge)
    idx(c->inc_pool, c->inc_top, 0, T * c->npe);               // incidence entries: element * nodes + local
    add(c->Gc, c->T0, 8);
    add(c->side, c->T0, 1);
    add(c->split_step, c->T0, 4);
    add(c->split_G, c->T0, 8);
    add(c->ud_tet, c->T0, 8);
    add(c->cand_flag, c->T0, 1);
    idx(c->cand_list, c->n_cand, 0, c->T0);
    idx(c->node_of_key, 2 * c->E0, 0, N, true);
    add(c->hkeys, c->hash_cap, 8);
    idx(c->hvals, c->hash_cap, 0, E, true);
    add(c->hfirst, c->hash_cap, 4);
    add(c->Ud, 1, 8);
    // node storage order (creation id of each stored node) and the node references a
    // renumbering rewrites besides conn and node_of_key
    idx(c->ext_of_int, N, 0, N);
    idx(c->oe_n0, c->E0, 0, N);
    idx(c->oe_n1, c->E0, 0, N);
    idx(c->dir_key, c->n_dir, 0, 4 * N);
    return f;
}

void header(const cem_ctx* c, int64_t h[HDR_COUNT]) {
    h[HDR_ELEM] = c->elem_type;
    h[HDR_PREC] = c->precision;
    h[HDR_N0] = c->N0;
    h[HDR_T0] = c->T0;
    h[HDR_E0] = c->E0;
    h[HDR_NC] = c->Nc;
    h[HDR_TC] = c->Tc;
    h[HDR_EC] = c->Ec;
    h[HDR_FANCAP] = c->fan_cap;
    h[HDR_INCCAP] = c->inc_cap;
    h[HDR_HASHCAP] = c->hash_cap;
    h[HDR_NINST] = c->n_inst;
    h[HDR_SPLITMODE] = c->split_mode;
    h[HDR_N] = c->N;
    h[HDR_T] = c->T;
    h[HDR_E] = c->E;
    h[HDR_NCAND] = c->n_cand;
    h[HDR_NSPLITALL] = c->n_split_all;
    h[HDR_NSPLITRUN] = c->n_split_run;
    h[HDR_NACTIVE] = c->n_active;
    h[HDR_FANTOP] = c->fan_top;
    h[HDR_INCTOP] = c->inc_top;
    h[HDR_STEP] = c->step;
    std::memcpy(&h[HDR_DT_BITS], &c->dt, sizeof(double));
    h[HDR_RENUMBERED] = c->renumbered ? 1 : 0;
    h[HDR_REORDER_N] = c->reorder_n;
    h[HDR_NREORDER] = c->n_reorder;
}

// The context's counts that a checkpoint sets (kept to restore them when a load fails).
struct Counts {
    int64_t N, T, E, n_cand, n_split_all, n_split_run, n_active, fan_top, inc_top, step, reorder_n, n_reorder;
    bool renumbered;
};

Counts counts_of(const cem_ctx* c) {
    return {c->N, c->T, c->E, c->n_cand, c->n_split_all, c->n_split_run, c->n_active, c->fan_top, c->inc_top,
            c->step, c->reorder_n, c->n_reorder, c->renumbered};
}

void set_counts(cem_ctx* c, const Counts& k) {
    c->N = k.N;
    c->T = k.T;
    c->E = k.E;
    c->n_cand = k.n_cand;
    c->n_split_all = k.n_split_all;
    c->n_split_run = k.n_split_run;
    c->n_active = k.n_active;
    c->fan_top = k.fan_top;
    c->inc_top = k.inc_top;
    c->step = k.step;
    c->reorder_n = k.reorder_n;
    c->n_reorder = k.n_reorder;
    c->renumbered = k.renumbered;
}

}  // namespace

extern "C" int cem_save(cem_ctx* c, const char* path) {
    if (!c || !path) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "cem_set_material must be called before cem_save");
    CEM_CK(c, cudaSetDevice(c->device));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return cem_fail(c, CEM_EINVAL, "cannot open the checkpoint file for writing");
    int64_t h[HDR_COUNT];
    header(c, h);
    bool ok = std::fwrite(TAG, 1, 8, fp) == 8 && std::fwrite(h, sizeof(int64_t), HDR_COUNT, fp) == HDR_COUNT;
    uint64_t hash = fnv1a(fnv1a(FNV_BASIS, TAG, 8), h, sizeof h);
    std::vector<char> buf;
    for (const Field& f : fields(c)) {
        if (!ok) break;
        buf.resize(f.bytes);
        if (cudaMemcpy(buf.data(), f.p, f.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(fp);
            return cem_fail(c, CEM_ECUDA, "device to host copy of the checkpoint");
        }
        const int64_t nb = (int64_t)f.bytes;
        ok = std::fwrite(&nb, sizeof nb, 1, fp) == 1 && std::fwrite(buf.data(), 1, f.bytes, fp) == f.bytes;
        hash = fnv1a(fnv1a(hash, &nb, sizeof nb), buf.data(), f.bytes);
    }
    ok = ok && std::fwrite(&hash, sizeof hash, 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? CEM_OK : cem_fail(c, CEM_EINVAL, "writing the checkpoint file failed");
}

extern "C" int cem_load(cem_ctx* c, const char* path) {
    if (!c || !path) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "cem_set_material must be called before cem_load");
    CEM_CK(c, cudaSetDevice(c->device));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    ++c->topo_version;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return cem_fail(c, CEM_EINVAL, "cannot open the checkpoint file");
    char tag[8];
    int64_t h[HDR_COUNT], mine[HDR_COUNT];
    if (std::fread(tag, 1, 8, fp) != 8 || std::memcmp(tag, TAG, 8) != 0 ||
        std::fread(h, sizeof(int64_t), HDR_COUNT, fp) != HDR_COUNT) {
        std::fclose(fp);
        return cem_fail(c, CEM_EINVAL, "not a checkpoint file");
    }
    header(c, mine);
    for (int q = HDR_ELEM; q <= HDR_SPLITMODE; ++q)
        if (h[q] != mine[q]) {
            std::fclose(fp);
            return cem_fail(c, CEM_EINVAL, "checkpoint of a different mesh, precision or capacity");
        }
    if (h[HDR_DT_BITS] != mine[HDR_DT_BITS]) {
        std::fclose(fp);
        return cem_fail(c, CEM_EINVAL, "checkpoint with a different time step (material)");
    }
    // counts within the context's capacities (the file is not trusted)
    const bool sizes_ok = h[HDR_N] >= c->N0 && h[HDR_N] <= c->Nc && h[HDR_T] >= c->T0 && h[HDR_T] <= c->Tc &&
                          h[HDR_E] >= c->E0 && h[HDR_E] <= c->Ec && h[HDR_NCAND] >= 0 && h[HDR_NCAND] <= c->T0 &&
                          h[HDR_FANTOP] >= 0 && h[HDR_FANTOP] <= c->fan_cap && h[HDR_INCTOP] >= 0 &&
                          h[HDR_INCTOP] <= c->inc_cap && h[HDR_NSPLITALL] >= 0 && h[HDR_NSPLITALL] <= c->S_cap &&
                          h[HDR_NSPLITRUN] >= 0 && h[HDR_NACTIVE] >= 0 && h[HDR_NACTIVE] <= h[HDR_T] &&
                          h[HDR_STEP] >= 0 && h[HDR_REORDER_N] >= 0 && h[HDR_REORDER_N] <= h[HDR_N] &&
                          h[HDR_NREORDER] >= 0 && (h[HDR_RENUMBERED] == 0 || h[HDR_RENUMBERED] == 1);
    if (!sizes_ok) {
        std::fclose(fp);
        return cem_fail(c, CEM_EINVAL, "checkpoint counts exceed the context's capacities");
    }
    // adopt the saved counts (they size the arrays), then read and hash the whole
    // file once before anything on the device changes
    const Counts old = counts_of(c);
    set_counts(c, {h[HDR_N], h[HDR_T], h[HDR_E], h[HDR_NCAND], h[HDR_NSPLITALL], h[HDR_NSPLITRUN], h[HDR_NACTIVE],
                   h[HDR_FANTOP], h[HDR_INCTOP], h[HDR_STEP], h[HDR_REORDER_N], h[HDR_NREORDER],
                   h[HDR_RENUMBERED] != 0});
    const std::vector<Field> fl = fields(c);
    const long data_at = std::ftell(fp);
    uint64_t hash = fnv1a(fnv1a(FNV_BASIS, tag, 8), h, sizeof h);
    bool ok = data_at >= 0;
    std::vector<char> buf;
    bool in_range = true;
    // the list offsets and counts and the storage order, kept for the cross checks below
    std::vector<int> keep_off[2], keep_cnt[2], keep_ext;
    for (size_t q = 0; q < fl.size() && ok; ++q) {
        int64_t nb = 0;
        ok = std::fread(&nb, sizeof nb, 1, fp) == 1 && nb == (int64_t)fl[q].bytes;
        if (!ok) break;
        hash = fnv1a(hash, &nb, sizeof nb);
        std::vector<int>* keep = fl[q].p == c->fan_off ? &keep_off[0] : fl[q].p == c->fan_cnt ? &keep_cnt[0]
                               : fl[q].p == c->inc_off ? &keep_off[1] : fl[q].p == c->inc_cnt ? &keep_cnt[1]
                               : fl[q].p == c->ext_of_int ? &keep_ext : nullptr;
        for (size_t done = 0; done < fl[q].bytes && ok;) {   // in pieces of at most 64 MiB (whole int32 entries)
            const size_t n = std::min(fl[q].bytes - done, (size_t)1 << 26);
            buf.resize(n);
            ok = std::fread(buf.data(), 1, n, fp) == n;
            if (ok) hash = fnv1a(hash, buf.data(), n);
            if (ok && fl[q].hi > 0) {
                const int* v = (const int*)buf.data();
                for (size_t k = 0; k < n / 4; ++k)
                    in_range = in_range && ((v[k] >= fl[q].lo && v[k] < fl[q].hi) || (fl[q].unset && v[k] == -1));
                if (keep) keep->insert(keep->end(), v, v + n / 4);
            }
            done += n;
        }
    }
    uint64_t want = 0;
    ok = ok && std::fread(&want, sizeof want, 1, fp) == 1 && want == hash;
    if (!ok) {
        set_counts(c, old);
        std::fclose(fp);
        return cem_fail(c, CEM_EINVAL, "checkpoint file truncated, inconsistent or corrupt; context unchanged");
    }
    // every list inside its pool's used part; the storage order a permutation of [0, N)
    const int64_t tops[2] = {c->fan_top, c->inc_top};
    for (int k = 0; k < 2 && in_range; ++k)
        for (size_t x = 0; x < keep_off[k].size() && x < keep_cnt[k].size(); ++x)
            in_range = in_range && (int64_t)keep_off[k][x] + keep_cnt[k][x] <= tops[k];
    if (in_range && !keep_ext.empty()) {
        std::vector<char> seen(keep_ext.size(), 0);
        for (int v : keep_ext) {
            in_range = in_range && !seen[v];
            seen[v] = 1;
        }
    }
    if (!in_range) {
        set_counts(c, old);
        std::fclose(fp);
        return cem_fail(c, CEM_EINVAL, "checkpoint holds an index out of range; context unchanged");
    }
    // node maps: identity, then the saved storage order of the first N nodes and its inverse
    if (int rc = cem_reorder_identity(c)) {
        std::fclose(fp);
        return rc;
    }
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    if (std::fseek(fp, data_at, SEEK_SET) != 0) {
        std::fclose(fp);
        return cem_fail(c, CEM_EINVAL, "checkpoint file cannot be re-read; context state undefined");
    }
    for (const Field& f : fl) {
        int64_t nb = 0;
        buf.resize(f.bytes);
        if (std::fread(&nb, sizeof nb, 1, fp) != 1 || nb != (int64_t)f.bytes ||
            std::fread(buf.data(), 1, f.bytes, fp) != f.bytes) {
            std::fclose(fp);
            return cem_fail(c, CEM_EINVAL, "checkpoint file changed while loading; context state undefined");
        }
        if (cudaMemcpy(f.p, buf.data(), f.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            std::fclose(fp);
            return cem_fail(c, CEM_ECUDA, "host to device copy of the checkpoint");
        }
    }
    std::fclose(fp);
    CEM_CK(c, cudaDeviceSynchronize());
    if (int rc = cem_reorder_inverse(c)) return rc;
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    return cem_refresh_act_orig(c);
}
