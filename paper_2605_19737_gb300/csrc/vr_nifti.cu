// vr_nifti.cu -- NIfTI-1 ingestion (Sec. 2.1: all volumes are provided in, or
// converted to, NIfTI-1). Host code only: parse the 348-byte header of a
// single-file .nii (either byte order), read the first 3D volume, apply the
// scl_slope / scl_inter intensity scaling, convert the spacing to mm, and hand
// the samples to vr_load_volume.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "vr_internal.cuh"

namespace {

struct NiftiHeader {
    int dims[3];
    int nt;          // volumes stored (only the first is read)
    int datatype;
    int bitpix;
    float spacing[3];  // mm
    float scl_slope, scl_inter;
    long vox_offset;
    bool swap;
};

template <class T>
T rd(const unsigned char* b, int off, bool swap) {
    unsigned char tmp[sizeof(T)];
    memcpy(tmp, b + off, sizeof(T));
    if (swap)
        for (size_t i = 0; i < sizeof(T) / 2; ++i) {
            const unsigned char t = tmp[i];
            tmp[i] = tmp[sizeof(T) - 1 - i];
            tmp[sizeof(T) - 1 - i] = t;
        }
    T v;
    memcpy(&v, tmp, sizeof(T));
    return v;
}

// 0 on success, else a message in err.
int parse_header(const unsigned char* b, NiftiHeader* h, char* err, size_t errlen) {
    int32_t sz = rd<int32_t>(b, 0, false);
    bool swap = false;
    if (sz != 348) {
        swap = true;
        sz = rd<int32_t>(b, 0, true);
        if (sz != 348) {
            snprintf(err, errlen, "not a NIfTI-1 header (sizeof_hdr != 348)");
            return 1;
        }
    }
    if (memcmp(b + 344, "n+1\0", 4) != 0) {
        snprintf(err, errlen, "only single-file NIfTI-1 (.nii, magic n+1) is supported");
        return 1;
    }
    const int16_t ndim = rd<int16_t>(b, 40, swap);
    if (ndim < 3 || ndim > 7) {
        snprintf(err, errlen, "dim[0] = %d: need a 3D or 4D volume", (int)ndim);
        return 1;
    }
    for (int a = 0; a < 3; ++a) h->dims[a] = rd<int16_t>(b, 42 + 2 * a, swap);
    h->nt = ndim >= 4 ? rd<int16_t>(b, 48, swap) : 1;
    if (h->nt < 1) h->nt = 1;
    h->datatype = rd<int16_t>(b, 70, swap);
    h->bitpix = rd<int16_t>(b, 72, swap);
    const int units = b[123] & 7;  // xyzt_units: 1 metre, 2 mm, 3 micron
    const float scale = units == 1 ? 1000.0f : (units == 3 ? 0.001f : 1.0f);
    for (int a = 0; a < 3; ++a) h->spacing[a] = fabsf(rd<float>(b, 80 + 4 * a, swap)) * scale;
    h->vox_offset = (long)rd<float>(b, 108, swap);
    h->scl_slope = rd<float>(b, 112, swap);
    h->scl_inter = rd<float>(b, 116, swap);
    h->swap = swap;
    if (h->vox_offset < 352) h->vox_offset = 352;
    return 0;
}

int bytes_of(int datatype) {
    switch (datatype) {
        case 2: case 256: return 1;     // uint8, int8
        case 4: case 512: return 2;     // int16, uint16
        case 8: case 768: case 16: return 4;  // int32, uint32, float32
        case 64: return 8;              // float64
        default: return 0;
    }
}

double sample(const unsigned char* p, int datatype, bool swap) {
    switch (datatype) {
        case 2: return (double)p[0];
        case 256: return (double)(int8_t)p[0];
        case 4: return (double)rd<int16_t>(p, 0, swap);
        case 512: return (double)rd<uint16_t>(p, 0, swap);
        case 8: return (double)rd<int32_t>(p, 0, swap);
        case 768: return (double)rd<uint32_t>(p, 0, swap);
        case 16: return (double)rd<float>(p, 0, swap);
        case 64: return rd<double>(p, 0, swap);
        default: return 0.0;
    }
}

int read_header(const char* path, NiftiHeader* h, char* err, size_t errlen) {
    FILE* f = fopen(path, "rb");
    if (!f) {
        snprintf(err, errlen, "cannot open %s", path);
        return 1;
    }
    unsigned char b[348];
    const size_t got = fread(b, 1, sizeof b, f);
    fclose(f);
    if (got != sizeof b) {
        snprintf(err, errlen, "%s: shorter than a NIfTI-1 header", path);
        return 1;
    }
    return parse_header(b, h, err, errlen);
}

}  // namespace

extern "C" {

vr_status vr_nifti_info(const char* path, int* h_dims, float* h_spacing, int* h_datatype) {
    if (!path) return VR_ERR_INVALID_ARG;
    NiftiHeader h;
    char err[256];
    if (read_header(path, &h, err, sizeof err)) return VR_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        if (h_dims) h_dims[a] = h.dims[a];
        if (h_spacing) h_spacing[a] = h.spacing[a];
    }
    if (h_datatype) *h_datatype = h.datatype;
    return VR_OK;
}

vr_status vr_load_nifti(vr_ctx* ctx, const char* path, int* vol_id) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (!path || !vol_id) return vr::set_error(ctx, VR_ERR_INVALID_ARG, "load_nifti: NULL pointer");
    NiftiHeader h;
    char err[256];
    if (read_header(path, &h, err, sizeof err)) return vr::set_error(ctx, VR_ERR_INVALID_ARG, err);
    const int bpv = bytes_of(h.datatype);
    if (!bpv || bpv * 8 != h.bitpix)
        return vr::set_error(ctx, VR_ERR_INVALID_ARG, "load_nifti: unsupported datatype/bitpix");
    for (int a = 0; a < 3; ++a)
        if (h.dims[a] < 2 || h.dims[a] > 2048)
            return vr::set_error(ctx, VR_ERR_INVALID_ARG, "load_nifti: dims outside [2, 2048]");
    const long long nvox = (long long)h.dims[0] * h.dims[1] * h.dims[2];
    std::vector<unsigned char> raw((size_t)nvox * bpv);
    FILE* f = fopen(path, "rb");
    if (!f) return vr::set_error(ctx, VR_ERR_INVALID_ARG, "load_nifti: cannot open file");
    const bool ok = fseek(f, h.vox_offset, SEEK_SET) == 0 && fread(raw.data(), 1, raw.size(), f) == raw.size();
    fclose(f);
    if (!ok) return vr::set_error(ctx, VR_ERR_INVALID_ARG, "load_nifti: file shorter than its header says");
    const bool scaled = h.scl_slope != 0.0f && !(h.scl_slope == 1.0f && h.scl_inter == 0.0f);
    if (h.datatype == 512 && !scaled && !h.swap)  // uint16 as stored: no conversion
        return vr_load_volume(ctx, raw.data(), 0, VR_U16, h.dims[0], h.dims[1], h.dims[2], h.spacing[0],
                              h.spacing[1], h.spacing[2], vol_id);
    std::vector<float> vals((size_t)nvox);
    for (long long i = 0; i < nvox; ++i) {
        double x = sample(raw.data() + (size_t)i * bpv, h.datatype, h.swap);
        if (scaled) x = x * h.scl_slope + h.scl_inter;
        vals[(size_t)i] = (float)x;
    }
    return vr_load_volume(ctx, vals.data(), 0, VR_F32, h.dims[0], h.dims[1], h.dims[2], h.spacing[0], h.spacing[1],
                          h.spacing[2], vol_id);
}

}  // extern "C"
