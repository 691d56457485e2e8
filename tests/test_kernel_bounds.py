"""Shared-memory bounds of the temporally blocked kernels, checked on the host.

The 1D cross-correlation kernel (csrc/xcorr.cu) stages a chunk plus a halo of sweeps x r cells per side in a
shared-memory buffer and runs the sweeps there.  This test reads the kernel's constants from
its source and restates its index ranges, then checks for every radius and sweep count the
host accepts:
* the staged span fits the buffer;
* every register-window read and every output write of every sweep stays in the buffer
  (int32 / FP32: 256 threads x 9 outputs from windows of 9 + 2r cells);
* one pass of the threads covers the whole valid span of every sweep;
* FP64 (one output per thread, runtime chunk length): the chunk is even and 256..2048, its
  buffers hold the staged span, and the launch fits in shared memory.
The sweep-count rule is restated too; the test fails if its source text changes, so the
restatement is updated with it.

The 2D heat kernel (csrc/diffusion2d_tb.cu) keeps per-warp rings of rows: its x-neighbour
reads, its prefetch slots and its ring depths are checked for K = 2, 4 and r = 1..4.

The wide cross-correlation and the max filter (csrc/xcorr_wide.cu) stage chunks by 1D bulk
copies: copy sizes and buffer starts are 16-byte multiples, and every read of the register
blocks and of the doubling passes stays in its buffer, for every accepted radius.

TMA: every tiled load of the heat and MHD kernels starts at an x coordinate whose byte
offset is a multiple of 16, with a box inner extent that is a multiple of 16 bytes, for every
dtype, tile width and radius; no kernel issues a tiled store.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "paper_2406_08923_gb300", "csrc", "xcorr.cu")).read()


def _const(name):
    m = re.search(r"constexpr int %s = ([^;]+);" % name, SRC)
    assert m, name
    expr = m.group(1).split("//")[0]
    env = {k: _const(k) for k in re.findall(r"\bXC_[A-Z_]+\b", expr)}
    return int(eval(expr, {"__builtins__": {}}, env))


T, V, MAXS, PAD = _const("XC_THREADS"), _const("XC_V"), _const("XC_MAX_SWEEPS"), _const("XC_PAD")
CHUNK, BUF = _const("XC_CHUNK"), _const("XC_BUF")
SMEM_MAX = 227 * 1024


def max_sweeps(r):
    # xcorr_max_sweeps_per_launch
    return MAXS if r <= 4 else min(MAXS, 1 + 60 // r)


def test_sweep_rule_source_is_the_restated_one():
    assert "return r <= 4 ? XC_MAX_SWEEPS : std::min(XC_MAX_SWEEPS, 1 + 60 / r);" in SRC
    assert (T, V, MAXS, PAD, CHUNK, BUF) == (256, 9, 16, 4, 2184, 2444)


def test_window_kernel_stays_in_its_buffers():
    # int32 and FP32 at r = 0..4; FP32 also at r = 5..32
    for r in range(0, 33):
        for sweeps in range(1, max_sweeps(r) + 1):
            H = sweeps * r
            W = CHUNK + 2 * H
            assert PAD + W <= BUF, (r, sweeps)  # staging writes buf[PAD + e], e < W
            for s in range(1, sweeps + 1):
                q_first, q_last = s * r, s * r + V * (T - 1)
                lo_read = PAD + q_first - r
                hi_read = PAD + q_last - r + (V + 2 * r) - 1
                hi_write = PAD + q_last + V - 1
                assert 0 <= lo_read and hi_read < BUF and hi_write < BUF, (r, sweeps, s)
                # the valid span [s r, W - s r) is covered by one pass of the threads
                assert W - s * r <= q_last + V, (r, sweeps, s)
            # the result read back: res[p] = src[PAD + H + p], p < CHUNK
            assert PAD + H + CHUNK - 1 < BUF


T64, F64_CAP, F64_MULTI = _const("XC_T64"), 4096, _const("XC_F64_MULTI_CHUNK")


def f64_launch(n, sms, l2=129 << 20):
    # run<double>: (chunk, threads).  Whole waves of 2 x 512-thread CTAs per SM (chunks up to
    # 4096, even, >= 256) while input and output fill at most 7/8 of L2, else 2048-cell
    # chunks in 256-thread CTAs
    wave = 2 * sms
    if 16 * n > l2 - l2 // 8:
        return F64_MULTI, T
    waves = max(1, (n + wave * F64_CAP - 1) // (wave * F64_CAP))
    per = (n + wave * waves - 1) // (wave * waves)
    return min(F64_CAP, max(256, (per + 1) & ~1)), T64


def f64_chunk(n, sms):
    return f64_launch(n, sms)[0]


def f64_stride(chunk, halo):
    # xc_f64_stride
    return (PAD + chunk + 2 * halo + 1) & ~1


def test_f64_chunks_and_buffers():
    assert "chunk_len = (int)std::min<int64_t>(chunk_len, std::max<int64_t>(256, (per + 1) & ~int64_t(1)));" in SRC
    assert "const int64_t waves = std::max<int64_t>(1, (g.n[0] + wave * chunk_len - 1) / (wave * chunk_len));" in SRC
    assert "wide = 2 * (int64_t)sizeof(T) * g.n[0] <= l2 - l2 / 8;" in SRC
    assert "const int64_t wave = 2 * (int64_t)device_sms();" in SRC
    assert "chunk_len = XC_F64_MULTI_CHUNK;" in SRC
    assert "return sizeof(T) == 8 ? 4096 : XC_CHUNK;" in SRC
    assert F64_MULTI == 2048
    assert "return (XC_PAD + chunk + 2 * halo + 1) & ~1;" in SRC
    assert T64 == 512
    sizes = [1, 7, 255, 256, 4099, 5003, 65536, 2 ** 20, 2 ** 20 + 1, 2 ** 21 + 5, 2 ** 22, 3 << 21, 2 ** 23,
             2 ** 24, 2 ** 26 + 3]
    for sms, l2 in ((132, 50 << 20), (148, 126 << 20), (152, 129 << 20), (152, 135 << 20), (160, 256 << 20),
                    (152, 0)):
        for n in sizes:
            c, nt = f64_launch(n, sms, l2)
            assert c % 2 == 0 and 256 <= c <= F64_CAP, (n, sms, c)
            per_sm = 1024 // nt
            blocks = (n + c - 1) // c
            assert blocks * c >= n and (blocks - 1) * c < n
            if nt == T64 and per_sm * sms * 256 <= n:
                # whole waves: the last wave is not more than one CTA per SM short
                waves = -(-blocks // (per_sm * sms))
                assert blocks > waves * per_sm * sms - sms, (n, sms, blocks, waves)
            for r in range(0, 5):
                for sweeps in range(1, max_sweeps(r) + 1):
                    H = sweeps * r
                    S = f64_stride(c, H)
                    W = c + 2 * H
                    assert S % 2 == 0 and PAD + W <= S  # second buffer 16-byte aligned; span fits
                    for s in range(1, sweeps + 1):
                        # p in [s r, W - s r), reads p + j for |j| <= r
                        assert PAD + (s - 1) * r >= 0 and PAD + W - (s - 1) * r <= S
                    assert per_sm * 2 * 8 * S <= SMEM_MAX  # CTAs per SM x two buffers
    # the 2^20-cell benchmark on 152 SMs: 3450-cell chunks, 304 CTAs of 512 threads, one wave;
    # 2^22 cells: 4 waves of 3450-cell chunks; 2^23 and 2^24 cells (more than L2 holds):
    # 2048-cell chunks of 256 threads
    assert f64_launch(2 ** 20, 152) == (3450, 512) and (2 ** 20 + 3449) // 3450 == 304
    assert f64_launch(2 ** 22, 152) == (3450, 512) and -(-2 ** 22 // 3450) == 1216
    assert f64_launch(3 << 21, 152) == (3450, 512)
    assert f64_launch(2 ** 23, 152) == (2048, 256) and f64_launch(2 ** 24, 152) == (2048, 256)
    assert f64_launch(2 ** 23, 152, 135 << 20) == (2048, 256)


def test_f64_rotated_rows_cover_the_span_once():
    # warp w starts at row k0 = (w - rot) mod NW and strides by NT cells: every cell of
    # [lo, hi) is computed by exactly one thread, for every rotation
    assert "int k0 = (int)(threadIdx.x >> 5) - rot;" in SRC
    assert "for (int p = lo + 32 * k0 + (int)(threadIdx.x & 31); p < hi; p += NT) {" in SRC
    assert "const int rot = (s + (int)blockIdx.x) % NW;" in SRC
    NW = T64 // 32
    for span in (1, 31, 32, 33, 511, 512, 513, 1726, 3450, 3510, 4096 + 128):
        for rot in range(NW):
            seen = [0] * span
            for t in range(T64):
                k0 = (t >> 5) - rot
                if k0 < 0:
                    k0 += NW
                p = 32 * k0 + (t & 31)
                while p < span:
                    seen[p] += 1
                    p += T64
            assert all(x == 1 for x in seen), (span, rot)


# ---------------------------------------------------------------------------------------------
# 2D temporally blocked heat kernel (csrc/diffusion2d_tb.cu): per-warp rings in shared memory.

TB_SRC = open(os.path.join(ROOT, "paper_2406_08923_gb300", "csrc", "diffusion2d_tb.cu")).read()


def tb_g(K, s, R):
    return tb_g(K, 1, R) + 1 if s == 0 else ((K - s) * R + 3) // 4


def test_blocked_2d_rings_stay_in_bounds():
    assert "return s == 0 ? tb_g(K, 1, R) + 1 : ((K - s) * R + 3) / 4;" in TB_SRC
    assert "constexpr int TB_WARPS = 4;" in TB_SRC
    for K in (2, 4):  # the step counts launch_diffusion2d_tb accepts
        for R in range(1, 5):
            G0, G1 = tb_g(K, 0, R), tb_g(K, 1, R)
            TXG, NQ = 32 - 2 * G1, 2 * R + 1
            W, NL, P = TXG + 2 * G0, 2 * NQ, min(3 * R + 1, 7)
            ring0, ringi = NL * W * 4, NQ * W * 4
            warp_floats = ring0 + (K - 1) * ringi
            assert TXG >= 8 and W <= 64 and P + R < NL, (K, R)
            assert 4 * warp_floats * 4 <= SMEM_MAX, (K, R)
            # f_0 fetch: a lane writes groups lane and (if lane + 32 < W) lane + 32 of its row
            assert max(lane + 32 * h for lane in range(32) for h in range(2) if lane + 32 * h < W) == W - 1
            for S in range(1, K + 1):
                GS = tb_g(K, S, R)
                active = TXG + 2 * GS
                assert active <= 32, (K, R, S)
                q = [lane - GS + G0 for lane in range(active)]
                # x neighbours: groups q - 1 .. q + 1 of the stage's input row
                assert min(q) - 1 >= 0 and max(q) + 1 <= W - 1, (K, R, S)
                # the row of stage S - 1 that stage S reads R rows later is still in its ring
                assert R < (NL if S == 1 else NQ)
            # prefetching row j + P overwrites row j + P - NL, older than the oldest row in use
            assert P - NL < -R


# ---------------------------------------------------------------------------------------------
# TMA tile loads (heat 2D/3D, MHD): the innermost coordinate of every tiled load, times the
# element size, is a multiple of 16 bytes, and so is the box's inner extent.

CSRC = os.path.join(ROOT, "paper_2406_08923_gb300", "csrc")


def _read(name):
    return open(os.path.join(CSRC, name)).read()


def test_tma_loads_start_on_16_byte_boundaries():
    api, common = _read("api.cu"), _read("common.cuh")
    # every TMA access is a load (no tiled store or reduce, so no negative store coordinates)
    tensor_ops = re.findall(r'"(cp\.async\.bulk\.tensor[^"]*)"', common)
    assert tensor_ops and all(".shared::cluster.global." in op for op in tensor_ops), tensor_ops
    # x origin of the padded layout: the radius rounded up to 16 bytes; rows padded to 32 bytes
    assert "const int64_t xoff = ((radius + v16 - 1) / v16) * v16;" in api
    assert "g.pad[0] = ((xoff + g.n[0] + xoff + align32 - 1) / align32) * align32;" in api
    # each kernel's load: x = off[0] + tile_x * TX - HX
    for f in ("diffusion.cu", "diffusion_f32.cu", "mhd.cu"):
        assert "const int bx = (int)g.off[0] + x0 - Cfg::HX" in _read(f), f
    assert "(int)g.off[0] + x0 - Cfg::HX" in _read("diffusion2d.cu")
    assert "static constexpr int HX = 4;" in _read("diffusion.cu")
    assert "TX = 128, HX = 4" in _read("diffusion_f32.cu")
    assert "TX = 32 * VX, HX = 4" in _read("diffusion2d.cu")
    assert "HX = 16 / (int)sizeof(S) >= 4 ? 16 / (int)sizeof(S) : 4;" in _read("mhd_rhs.cuh")
    families = []  # (esize, HX, tile widths, radii)
    families.append((8, 4, [64, 128], range(1, 5)))            # 3D heat FP64 (TX = 64 VP)
    families.append((4, 4, [128], range(1, 5)))                 # 3D heat FP32
    families += [(e, 4, [32 * vx for vx in (1, 2, 4)], range(1, 5)) for e in (4, 8)]  # 2D heat
    families += [(e, max(16 // e, 4), [16, 32, 64], [3]) for e in (8, 4, 2)]          # MHD
    for esize, hx, txs, radii in families:
        for r in radii:
            assert hx >= r  # the x halo in shared memory covers the stencil
            v16 = 16 // esize
            xoff = (r + v16 - 1) // v16 * v16
            for tx in txs:
                assert (tx + 2 * hx) * esize % 16 == 0, (esize, tx)  # box inner extent
                for tile in range(4):
                    x = xoff + tile * tx - hx
                    assert x * esize % 16 == 0, (esize, hx, tx, r, tile)
                for n in (7, 8, 100, 256, 383):
                    pad = (2 * xoff + n + 32 // esize - 1) // (32 // esize) * (32 // esize)
                    assert pad * esize % 32 == 0 and pad >= xoff + n + r


# ---------------------------------------------------------------------------------------------
# Wide cross-correlation and max filter (csrc/xcorr_wide.cu): bulk-copied staging buffers.

WIDE_SRC = _read("xcorr_wide.cu")


def _roundup(a, m):
    return (a + m - 1) // m * m


def test_wide_kernels_stay_in_their_buffers():
    for text in ("constexpr int WT = 256;", "constexpr int MF_CHUNK = 4096;",
                 "constexpr int WIDE_V_F32[] = {9, 11, 13, 15};", "constexpr int WIDE_V_F64[] = {5, 7, 9};",
                 "return (2 * rr(r) + CH + nwp(r) + V + L - 1) / L * L;", "return (2 * r + 1 + V - 1) / V * V;",
                 "return (MF_CHUNK + 2 * rr(r) + L - 1) / L * L;", "inline int maxf_nbuf(int r) { return r == 0 ? 2 : 1; }"):
        assert text in WIDE_SRC, text
    wt, mf = 256, 4096
    # cross-correlation: FP32 at r = 33..1024, FP64 at r = 5..1024
    for esize, vs, radii in ((4, (9, 11, 13, 15), range(33, 1025)), (8, (5, 7, 9), range(5, 1025))):
        L = 16 // esize
        for V in vs:
            ch = wt * V
            assert ch * esize % 16 == 0  # chunk starts c * CH stay 16-byte aligned
            for r in radii:
                rr, nwp = _roundup(r, L), _roundup(2 * r + 1, V)
                be, wlen = _roundup(2 * rr + ch + nwp + V, L), _roundup(nwp, L)
                assert be % L == 0 and wlen % L == 0  # every buffer starts 16-byte aligned
                assert (ch + 2 * rr) * esize % 16 == 0 and ch + 2 * rr <= be  # the bulk copy
                lead, span = rr - r, ch + 2 * r
                assert lead + span + (rr - r) - 1 < be  # zeroed tail past the span
                # reads s[base + j0 + q]: base <= (WT-1) V, j0 <= nwp - V, q <= 2V - 2
                assert lead + (wt - 1) * V + (nwp - V) + (2 * V - 2) < be
                assert esize * (wlen + be) <= SMEM_MAX  # one staging buffer always fits
    # max filter: int32 / FP32 / FP64 at r = 0..1024, nbuf staging buffers + 1 work buffer
    for esize in (4, 8):
        L = 16 // esize
        for r in range(0, 1025):
            rr = _roundup(r, L)
            be = _roundup(mf + 2 * rr, L)
            lead, span, w = rr - r, mf + 2 * r, 2 * r + 1
            assert (mf + 2 * rr) * esize % 16 == 0 and mf + 2 * rr <= be
            assert lead + span - 1 < be
            length = 1
            while 2 * length <= w:
                assert (span - 2 * length) + length < span  # a[i + len], i <= span - 2 len
                length *= 2
            assert (mf - 1) + (w - length) <= span - length  # the last read is a defined run
            nbuf = 2 if r == 0 else 1
            assert (nbuf + 1) * be * esize <= SMEM_MAX


# ---------------------------------------------------------------------------------------------
# MHD (csrc/mhd.cu): every variant's plane ring fits the shared memory of one CTA, and its
# threads fit the register file at the register count its launch bounds allow.


def test_mhd_variants_fit_shared_memory_and_registers():
    src = _read("mhd_rhs.cuh")
    for text in ("static constexpr int TXP = TX + 2 * HX;", "static constexpr int ROWS = TY + 2 * R6;",
                 "static constexpr int FIELD_ELEMS = ((TXP * ROWS * (int)sizeof(S) + 127) / 128) * 128 / (int)sizeof(S);",
                 "static constexpr int SLOT_ELEMS = 8 * FIELD_ELEMS;",
                 "static constexpr size_t SMEM = (size_t)NSLOT * SLOT_ELEMS * sizeof(S) + 128;"):
        assert text in src, text
    tables = _read("mhd.cu")
    for esize, macro in ((8, "MHD_VARIANTS_F64"), (4, "MHD_VARIANTS_F32"), (2, "MHD_VARIANTS_BF16")):
        line = re.search(r"#define " + macro + r"\(X\)(.*)", tables).group(1)
        variants = [tuple(int(v) for v in m) for m in re.findall(r"X\((\d+), (\d+), (\d+), (\d+)\)", line)]
        assert variants, macro
        hx = max(16 // esize, 4)
        for tx, ty, nslot, minb in variants:
            field = ((tx + 2 * hx) * (ty + 6) * esize + 127) // 128 * 128
            smem = nslot * 8 * field + 128
            assert smem <= SMEM_MAX, (macro, tx, ty, smem)
            assert minb * (smem + 64 + 1024) <= 233472, (macro, tx, ty, minb)  # CTAs per SM
            threads = tx * ty
            assert threads <= 1024 and threads % 32 == 0
            assert 65536 // (threads * minb) >= 64, (macro, tx, ty)  # registers per thread


# ---------------------------------------------------------------------------------------------
# Norms pass 1 (csrc/norms.cu): each warp walks its pieces with carried (segment, y, z) steps
# instead of dividing every piece index; the walk must visit exactly the pieces a division gives.

NORM_SRC = open(os.path.join(ROOT, "paper_2406_08923_gb300", "csrc", "norms.cu")).read()


def test_norms_piece_walk_matches_division():
    for text in ("const int64_t row = gw / segs, drow = nw / segs;", "sg = gw - row * segs;",
                 "dsg = nw - drow * segs;", "if (sg >= segs) { sg -= segs; carry = 1; }",
                 "y += dy + carry;  // dy < n1 and carry <= 1: at most one wrap",
                 "if (y >= n1) { y -= n1; z += 1; }",
                 "for (int64_t piece = gw; piece < pw.pieces; piece += nw, pw.next()) {"):
        assert text in NORM_SRC, text
    seg = 32 * 8 * 8
    assert "constexpr int NORM_SEG = 32 * NORM_U * 8;" in NORM_SRC
    for nx, ny, nz in ((256, 256, 4), (1, 1, 1), (2 ** 20, 1, 1), (5000, 3, 7), (2049, 17, 2), (13, 11, 9)):
        segs = -(-nx // seg)
        pieces = segs * ny * nz
        for nw in (1, 7, 2432, 4864):
            for gw in sorted({0, 1, nw // 2, nw - 1}):
                if gw >= nw:
                    continue
                row, drow = gw // segs, nw // segs
                sg, y, z = gw - row * segs, row % ny, row // ny
                dsg, dy, dz = nw - drow * segs, drow % ny, drow // ny
                piece = gw
                while piece < pieces:
                    r = piece // segs
                    assert (sg, y, z) == (piece - r * segs, r % ny, r // ny), (nx, ny, nz, nw, gw, piece)
                    piece += nw
                    sg += dsg
                    carry = 0
                    if sg >= segs:
                        sg, carry = sg - segs, 1
                    y += dy + carry
                    z += dz
                    if y >= ny:
                        y, z = y - ny, z + 1
