"""DLIC oracle: test infrastructure only.

A plain, slow CPU restatement of the coding method (dlic_oracle.c, loaded with
ctypes) and an FP64 reference of the training loss and its gradient
(train64.py).  Only the tests, the smoke check and the bench's CPU-baseline
leg use this package; the CUDA library never imports or links it.
"""
from .coder import (build, lib, encode, decode, symbol_tables, pixel_table, logits,
                    table_from_logits, gather, gather_window, rans_enc_step, rans_dec_step, fnv1a64,
                    max_encoded_bytes, gather_window3, encode_volume, decode_volume, symbols)

__all__ = ["build", "lib", "encode", "decode", "symbol_tables", "pixel_table", "logits",
           "table_from_logits", "gather", "gather_window", "rans_enc_step", "rans_dec_step", "fnv1a64",
           "max_encoded_bytes", "gather_window3", "encode_volume", "decode_volume", "symbols"]
