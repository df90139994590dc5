"""The checkpoint file's reader (pxsne_load) on the CPU: a file is checked --
magic, version, sizes, length and checksum -- before any device work, so a
damaged file is refused with PXSNE_E_ARG and a reason, and *out stays NULL.
The files are written here from the layout the header documents."""
import ctypes
import struct

import numpy as np
import pytest

import paper_1611_02568_gb300 as px

PXSNE_E_ARG, PXSNE_E_CUDA, PXSNE_E_UNSUPPORTED = -1, -3, -6


def fnv_words(payload: bytes) -> int:
    h = 14695981039346656037
    pad = (-len(payload)) % 8
    b = payload + b"\0" * pad
    for (w,) in struct.iter_unpack("<Q", b):
        h ^= w
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def make_file(n=4, version=1, magic=b"PXSNECK\0", corrupt=None, trailing=b"", short=0):
    p = px.Params(log2_r=4, k=1, perplexity=1.0)
    cp = bytes(p.c())
    assert len(cp) == 72
    rp = np.array([0, 1, 2, 3, 4], np.int64)[: n + 1]
    col = np.array([1, 0, 3, 2], np.int32)
    val = np.full(4, 0.25, np.float32)
    z = np.arange(2 * n, dtype=np.uint32) * np.uint32(123456789)
    u = np.zeros(2 * n, np.float32)
    g = np.ones(2 * n, np.float32)
    payload = b"".join(a.tobytes() for a in (rp, col, val, z, u, g))
    ck = fnv_words(payload)
    if corrupt is not None:
        payload = bytearray(payload)
        payload[corrupt] ^= 1
        payload = bytes(payload)
    head = magic + struct.pack("<II", version, 144) + cp
    head += struct.pack("<qqii", n, 4, 7, 0) + struct.pack("<dd", 2.0 ** -30, 2.0 ** -31)
    head += struct.pack("<QQ", len(rp) * 8 + 8 * 4 + 24 * n, ck)
    assert len(head) == 144
    data = head + payload + trailing
    return data[: len(data) - short] if short else data


@pytest.fixture(scope="module")
def lib():
    from paper_1611_02568_gb300 import build
    build.build()
    return px.load()


def _load(lib, path):
    h = ctypes.c_void_p(1)
    rc = lib.pxsne_load(ctypes.byref(h), str(path).encode(), None)
    return rc, h.value, lib.pxsne_last_error(None).decode()


def test_format_checksum_is_fnv1a_over_words():
    # FNV-1a's published 64-bit parameters: empty input gives the offset basis
    assert fnv_words(b"") == 14695981039346656037
    # one word: (basis ^ w) * prime mod 2^64
    w = 0x0102030405060708
    assert fnv_words(struct.pack("<Q", w)) == ((14695981039346656037 ^ w) * 1099511628211) % 2 ** 64
    # a partial last word is zero-padded
    assert fnv_words(b"\x01") == fnv_words(struct.pack("<Q", 1))


@pytest.mark.parametrize("case,code,reason", [
    (dict(corrupt=40), PXSNE_E_ARG, "checksum"),
    (dict(magic=b"PXSNECX\0"), PXSNE_E_ARG, "not a checkpoint"),
    (dict(version=2), PXSNE_E_UNSUPPORTED, "version"),
    (dict(short=5), PXSNE_E_ARG, "truncated"),
    (dict(trailing=b"\0"), PXSNE_E_ARG, "trailing"),
])
def test_damaged_files_are_refused_before_device_work(lib, tmp_path, case, code, reason):
    path = tmp_path / "ck.bin"
    path.write_bytes(make_file(**case))
    rc, h, msg = _load(lib, path)
    assert rc == code and h is None and reason in msg, (rc, msg)


def test_missing_file_and_null_arguments(lib, tmp_path):
    rc, h, msg = _load(lib, tmp_path / "absent.bin")
    assert rc == PXSNE_E_ARG and h is None and "cannot open" in msg
    assert lib.pxsne_load(None, b"x", None) == PXSNE_E_ARG
    assert lib.pxsne_save(None, b"x") == PXSNE_E_ARG


def test_a_sound_file_passes_the_checks(lib, tmp_path):
    # without a GPU the load stops at the device (PXSNE_E_CUDA); with one it
    # succeeds
    path = tmp_path / "ck.bin"
    path.write_bytes(make_file())
    rc, h, msg = _load(lib, path)
    assert rc in (0, PXSNE_E_CUDA), (rc, msg)
    if rc == 0:
        lib.pxsne_destroy(ctypes.c_void_p(h))
