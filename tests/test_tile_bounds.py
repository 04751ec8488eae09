"""Shared-memory bounds of the pipelined FP32 FFT kernels, checked on the CPU.

For every padded length L the launchers instantiate (64 ... 2048), the tile
width each launcher picks and, at L = 256 ... 1024, each launch variant of the
Y and Z kernels (8-column tiles; a split with a doubled first radix), every
shared-memory index the kernels form
(staged inputs, the exchange between the two DFT stages, the spectrum slice,
the twiddle table) is enumerated over all threads and loop indices and must
stay inside its buffer, and each CTA's shared memory must fit in 227 KB.  The
bulk-copy staging of the FP32 Z kernel is checked against the alignment and
size rules of the copies it issues.

The tile shapes below restate passes.cuh (Tile), common.cuh (Split) and
passes_impl.cuh (ZPipe, YPipe, YInvPipe, XFwdPipe, XInvPipe, the launchers'
tile widths, the kernels' index expressions); test_sources_still_define_*
fails if one of those lines changes, so that this restatement is updated with
it."""

import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_04691_gb300", "csrc")
SMEM_MAX = 227 * 1024            # dynamic shared memory per CTA (bytes)
CB = 8                           # complex64
LS = [64, 128, 256, 512, 1024, 2048]


def split(L):
    lg = int(L).bit_length() - 1
    L1 = 1 << ((lg + 1) // 2)
    return L1, L // L1


def tile(L, C, L1=None):
    L1, L2 = split(L) if L1 is None else (L1, L // L1)
    PK, PKI = L2 + 1, L1 + 1
    PC, PCI = (L1 * PK) | 1, (L2 * PKI) | 1
    return dict(L1=L1, L2=L2, NT=C * L2, PK=PK, PC=PC, PKI=PKI, PCI=PCI, SE=max(C * PC, C * PCI))


def yz_cols(L):                  # Y and Z launchers (FP32)
    return 8 if L > 1024 else 16


def yz_variants(L):              # (C, L1) of each launch variant (has_pipe_variants)
    L1 = split(L)[0]
    if 256 <= L <= 1024:
        return [(16, L1), (8, L1), (16, 2 * L1)]
    return [(yz_cols(L), L1)]


YZ = [(L, C, L1) for L in LS for C, L1 in yz_variants(L)]


def x_cols(L):                   # xpipe_cols<L>()
    want = max(1, 256 // split(L)[1])
    return max(1, want // 2)


def grid(*ranges):
    return np.meshgrid(*[np.arange(r) for r in ranges], indexing="ij")


@pytest.mark.parametrize("L,C,L1v", YZ)
def test_zconv_pipe_indices(L, C, L1v):
    t = tile(L, C, L1v)
    assert t["L1"] >= t["L2"] and 16 % C == 0                       # NI >= 1; C divides the spectrum group
    L1, L2, NT, PK, PC, PKI, PCI = (t[k] for k in ("L1", "L2", "NT", "PK", "PC", "PKI", "PCI"))
    E, S, TW = t["SE"], (L // 2 + 1) * C, L
    assert (E + S + TW) * CB <= SMEM_MAX
    tid, j1 = grid(NT, L1 // 2)
    c, jl = tid % C, tid // C
    j = j1 * L2 + jl
    assert (j * C + c)[j < L // 2].max() < S                       # staged input rows (n_in <= L/2)
    tid, k1 = grid(NT, L1)
    c, jl = tid % C, tid // C
    assert (c * PC + k1 * PK + jl).max() < E                         # forward exchange store
    assert (jl + k1 * L2).max() < TW
    s, j = grid(NT * (L1 // L2), L2)
    c2, k1 = s % C, s // C
    assert (c2 * PC + k1 * PK + j).max() < E                         # forward exchange load
    assert (k1 * L2 + j).max() < TW
    assert (c2 * PCI + j * PKI + k1).max() < E                       # inverse exchange store
    s, k2 = grid(NT * (L1 // L2), L2)
    c2, k1 = s % C, s // C
    lo = (k1 + k2 * L1)[k2 < L2 // 2]
    hi = (L - k1 - k2 * L1)[k2 >= L2 // 2]
    rows = np.concatenate([lo, hi])
    assert rows.min() >= 0 and rows.max() <= L // 2                 # the spectrum slice holds L/2 + 1 rows
    tid, k1 = grid(NT, L1)
    c, jl = tid % C, tid // C
    assert (c * PCI + jl * PKI + k1).max() < E                       # inverse exchange load


TMA_YZ = [(L, C, L1v) for L, C, L1v in YZ if C == 16 and L <= 1024]


@pytest.mark.parametrize("L,C,L1v", TMA_YZ)
def test_zconv_bulk_copy_staging(L, C, L1v):
    """The bulk-copy (TMA) staging of the FP32 Z kernel with 16-column tiles:
    every copy starts and ends on the boundaries the hardware requires, the
    boxes of input rows end inside the staging buffer for every n <= L/2, and
    the bytes a barrier phase expects stay below the transaction-count limit."""
    t = tile(L, C, L1v)
    E, S, TW = t["SE"], (L // 2 + 1) * C, L
    assert (E * CB) % 128 == 0                                        # S 128-byte aligned after E
    assert ((E + S + TW) * CB) % 8 == 0                              # the mbarrier after TW
    assert (E + S + TW) * CB + 128 + 16 <= SMEM_MAX                  # + alignment slack and barrier
    zbox = min(L // 2, 256)
    assert zbox <= 256 and C <= 256 and (C * CB) % 16 == 0           # box limits; inner extent
    H = L // 2 + 1
    for n in range(1, L // 2 + 1):
        nbox = -(-n // zbox)
        assert nbox * zbox <= L // 2 + 1                              # zero-filled rows stay in S
        assert nbox * zbox * C * CB < 1 << 20                         # expect_tx limit
        for q in range(nbox):
            assert (q * zbox * C * CB) % 128 == 0                     # destination of box q
        strides = [L * CB, L * L * CB, n * L * L * CB]                # tensor map strides
        assert all(st % 16 == 0 and st < 1 << 40 for st in strides)
    cb = np.arange(L // C)
    assert np.all((cb * C * CB) % 16 == 0)                            # x coordinate x element size
    ghat_bytes = (L // 2 + 1) * C * CB
    assert ghat_bytes % 16 == 0 and ghat_bytes < 1 << 20
    my = np.arange(H)[:, None]
    off = ((my * (L // 16) + cb[None, :]) * (L // 2 + 1) * 16 * CB)
    assert np.all(off % 16 == 0) and (H * H * L * CB) % 16 == 0        # spectrum source, per wave number


@pytest.mark.parametrize("L,C,L1v", YZ)
def test_yfwd_pipe_indices(L, C, L1v):
    t = tile(L, C, L1v)
    L1, L2, NT, PK, PC = (t[k] for k in ("L1", "L2", "NT", "PK", "PC"))
    E, S = t["SE"], (L // 2) * C
    assert (E + S + L) * CB <= SMEM_MAX
    tid, j1 = grid(NT, L1 // 2)
    c, jl = tid % C, tid // C
    j = j1 * L2 + jl
    assert (j * C + c)[j < L // 2].max() < S
    tid, k1 = grid(NT, L1)
    assert ((tid % C) * PC + k1 * PK + tid // C).max() < E
    s, j = grid(NT * (L1 // L2), L2)
    assert ((s % C) * PC + (s // C) * PK + j).max() < E


@pytest.mark.parametrize("L,C,L1v", YZ)
def test_yinv_pipe_indices(L, C, L1v):
    t = tile(L, C, L1v)
    L1, L2, NT, PKI, PCI = (t[k] for k in ("L1", "L2", "NT", "PKI", "PCI"))
    BUF = max(C * L, t["SE"])
    assert (BUF + L) * CB <= SMEM_MAX
    j, cc = grid(L, C)
    assert (j * C + cc).max() < BUF                                   # staged tile: L rows of C columns
    s, k2 = grid(NT * (L1 // L2), L2)
    c2, k1 = s % C, s // C
    assert ((k1 + L1 * k2) * C + c2).max() < BUF
    assert (c2 * PCI + k2 * PKI + k1).max() < BUF                    # exchange store (k2 plays ja)
    tid, k1 = grid(NT, L1)
    assert ((tid % C) * PCI + (tid // C) * PKI + k1).max() < BUF


@pytest.mark.parametrize("L", LS)
def test_xfwd_pipe_indices(L):
    C = x_cols(L)
    t = tile(L, C)
    L1, L2, NT, PK, PC = (t[k] for k in ("L1", "L2", "NT", "PK", "PC"))
    STAGE = 3 * C * (L // 2)
    assert (t["SE"] + STAGE + L) * CB <= SMEM_MAX
    tid, j1 = grid(NT, L1 // 2)
    j2, c = tid % L2, tid // L2
    j = j1 * L2 + j2
    assert (c * (L // 2) + j)[j < L // 2].max() < STAGE // 3       # r, p, s of C lines of n <= L/2
    tid, k1 = grid(NT, L1)
    assert ((tid // L2) * PC + k1 * PK + tid % L2).max() < t["SE"]
    s, j = grid(NT * (L1 // L2), L2)
    assert ((s // L1) * PC + (s % L1) * PK + j).max() < t["SE"]


@pytest.mark.parametrize("L", LS)
def test_xinv_pipe_indices(L):
    C = x_cols(L)
    t = tile(L, C)
    L1, L2, NT, PKI, PCI = (t[k] for k in ("L1", "L2", "NT", "PKI", "PCI"))
    BUF, EPI = max(C * L, t["SE"]), 2 * C * (L // 2)
    assert (BUF + EPI) * CB + 32 * 16 + 4 <= SMEM_MAX                # plus the static reduction scratch
    s, k2 = grid(NT * (L1 // L2), L2)
    c2, k1 = s // L1, s % L1
    assert (c2 * L + k1 + L1 * k2).max() < BUF
    assert (c2 * PCI + k2 * PKI + k1).max() < BUF
    tid, k1 = grid(NT, L1)
    assert ((tid // L2) * PCI + (tid % L2) * PKI + k1).max() < BUF
    tid, jb = grid(NT, L1 // 2)
    x = tid % L2 + L2 * jb
    assert ((tid // L2) * (L // 2) + x)[x < L // 2].max() < EPI // 2


def _read(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


@pytest.mark.parametrize("name,lines", [
    ("common.cuh", ["static constexpr int L1 = 1 << ((lg + 1) / 2);",
                    "static constexpr int L2 = L / L1;"]),
    ("passes.cuh", ["constexpr bool has_pipe_variants(int L) { return L >= 256 && L <= 1024; }",
                    "template <int L, int C, class T, int L1X = Split<L>::L1>",
                    "static constexpr int L1 = L1X;",
                    "static constexpr int L2 = L / L1X;",
                    "static constexpr int NT = C * L2;",
                    "static constexpr int PK = L2 + 1;",
                    "static constexpr int PC = (L1 * PK) | 1;",
                    "static constexpr int PKI = L1 + 1;",
                    "static constexpr int PCI = (L2 * PKI) | 1;",
                    "static constexpr int SMEM_ELEMS = (C * PC > C * PCI) ? C * PC : C * PCI;"]),
    ("passes_impl.cuh", ["constexpr int want = 256 / Split<L>::L2;",
                         "constexpr int c = lines_contig_f32<L>() / 2;",
                         "static constexpr int STAGE = 3 * C * (L / 2);",
                         "static constexpr int EPI = 2 * C * (L / 2);",
                         "static constexpr int BUF = (C * L > TL::SMEM_ELEMS) ? C * L : TL::SMEM_ELEMS;",
                         "static constexpr size_t S_ELEMS = size_t(L / 2 + (GZ ? 1 : 0)) * C;",
                         "static constexpr size_t S_ELEMS = size_t(L / 2) * C;",
                         "constexpr int C = L > 1024 ? 8 : 16;",
                         "constexpr int C = (L > 1024 && sizeof(T) == 4) ? 8 : 128 / int(sizeof(cpx<T>));",
                         "constexpr int C = xpipe_cols<L>();",
                         "cudaError_t e = Launch<T, L, 16, L1>::run(a, s, true, sm_count);",
                         "if (e == cudaSuccess) e = Launch<T, L, 8, L1>::run(a, s, true, sm_count);",
                         "if (e == cudaSuccess) e = Launch<T, L, 16, 2 * L1>::run(a, s, true, sm_count);",
                         "if (a.variant == 1) return Launch<T, L, 8, L1>::run(a, s, false, sm_count);",
                         "if (a.variant == 2) return Launch<T, L, 16, 2 * L1>::run(a, s, false, sm_count);",
                         "return Launch<T, L, 16, L1>::run(a, s, false, sm_count);",
                         "if (j < a.n_in) r[j1] = S[j * C + c];",
                         "E[c * PC + k1 * PK + jl] = r[k1];",
                         "b[it][j] = E[c2 * PC + k1 * PK + j];",
                         "const cpx<T>* lo = S + k1 * C + c2;",
                         "const cpx<T>* hi = S + (L - k1) * C + c2;",
                         "E[c2 * PCI + ja * PKI + k1] = b[it][ja];",
                         "r[k1] = E[c * PCI + jl * PKI + k1];",
                         "b[it][k2] = B[(k1 + L1 * k2) * C + c2];",
                         "B[c2 * PCI + j * PKI + k1] = b[it][j];",
                         "r[k1] = B[c * PCI + ja * PKI + k1];",
                         "b[it][k2] = okl ? B[c2 * L + k1 + L1 * k2] : czero<T>();",
                         "E[c * PC + k1 * PK + j2] = r[k1];",
                         "static constexpr bool TMA = GZ && C == kZGroup;",
                         "static constexpr size_t TMA_BYTES = TMA ? 128 + 16 : 0;",
                         "for (int q = 0; q < nbox; ++q) tma_load_4d(S + q * a.zbox * C, &a.zrows, cb * C, ky, q * a.zbox, rhs, bar);",
                         "constexpr unsigned bytes = unsigned(L / 2 + 1) * C * unsigned(sizeof(cpx<float>));",
                         "if constexpr (ZP::TMA) base += (128u - (smem_addr(smraw) & 127u)) & 127u;"]),
    ("ori_api.cu", ["const int zbox = std::min(L / 2, 256);",
                    "const cuuint32_t box[4] = {cuuint32_t(kZGroup), 1, cuuint32_t(zbox), 1};",
                    "if (enc != nullptr && L >= 64 && L <= 1024 && (reinterpret_cast<uintptr_t>(p->T2f) & 15u) == 0) {"]),
])
def test_sources_still_define_the_restated_shapes(name, lines):
    src = _read(name)
    for line in lines:
        assert line in src, f"{name} no longer contains: {line}"
