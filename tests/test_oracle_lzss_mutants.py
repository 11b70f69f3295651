"""Mutation check of the LZSS oracle's pins.

Each case copies ``oracle/lzss_oracle.c``, plants one plausible mistake (a
reversed tie-break, no overlapping sources, an off-by-one in a token field,
a shifted dictionary, a weakened rule), builds it with the unchanged Huffman
oracle into a temporary library, routes the ``oracle`` module to it and runs
the pins of ``test_oracle_lzss.py``.  Every mutant must fail at least one
pin.  The mistakes stay in the temporary copy, and every mutant keeps the
oracle's memory accesses within the buffers it is given.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_lzss as pins

_DIR = os.path.dirname(oracle.__file__)

MUTANTS = [
    ("ties_keep_largest_distance", "if (l > best_len) {", "if (l >= best_len) {"),
    ("no_overlapping_source", "while (l < maxlen &&", "while (l < maxlen && l < d &&"),
    ("length_field_plus_one", "(uint32_t)(best_len - P->min_len), len_bits(P)",
     "(uint32_t)(best_len - P->min_len + 1), len_bits(P)"),
    ("offset_field_is_distance", "(uint32_t)(best_d - 1), off_bits(P)",
     "(uint32_t)(best_d), off_bits(P)"),
    ("dictionary_shifted_one_byte", "((((j >> 3) & 255) >> (7 - (j & 7))) & 1)",
     "(((((j >> 3) + 1) & 255) >> (7 - (j & 7))) & 1)"),
    ("minimum_length_exclusive", "if (best_len >= P->min_len) { /* Z5",
     "if (best_len > P->min_len) { /* Z5"),
    ("literal_bits_reversed", "put_bits(&w, (uint32_t)data_bit(x, p + i), 1);",
     "put_bits(&w, (uint32_t)data_bit(x, p + k - 1 - i), 1);"),
    ("segments_not_aligned", "const uint64_t used = al16((bits + 7) / 8);",
     "const uint64_t used = (bits + 7) / 8;"),
    ("decode_ignores_stream_end", "return r.pos == code_bits ? ORACLE_OK : ORACLE_ERR_CORRUPT;",
     "return ORACLE_OK;"),
]


def _pin_list():
    out = [lambda nm=nm: pins.test_golden(nm) for nm in pins.golden_names()]
    out += [lambda p=p: pins.test_token_audit_random_inputs(p) for p in pins.PARAMS]
    out += [pins.test_zeros_closed_form, pins.test_container_layout,
            pins.test_container_edge_sizes_and_corruption]
    out += [lambda g=g: pins.test_round_trip(g, oracle.PAPER_LZSS)
            for g in ("bitstream", "zeros")]
    return out


def _build(tmp_path, name, old, new):
    src = open(os.path.join(_DIR, "lzss_oracle.c")).read()
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    d = tmp_path / name
    d.mkdir()
    (d / "lzss_oracle.c").write_text(src.replace(old, new))
    for f in ("huff_oracle.c", "huff_oracle.h"):
        (d / f).write_text(open(os.path.join(_DIR, f)).read())
    so = d / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", str(so),
                           str(d / "huff_oracle.c"), str(d / "lzss_oracle.c")])
    return str(so)


def test_unmutated_copy_passes_every_pin(tmp_path):
    so = _build(tmp_path, "identity", "if (l > best_len) {", "if (l > best_len) {")
    with oracle.use_library(so):
        for pin in _pin_list():
            pin()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(tmp_path, name, old, new):
    so = _build(tmp_path, name, old, new)
    caught = None
    with oracle.use_library(so):
        for pin in _pin_list():
            try:
                pin()
            except AssertionError as e:
                caught = e
                break
    assert caught is not None, f"mutant {name} passes every pin"
