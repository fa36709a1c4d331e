"""FP64 CPU oracle for SAAMG-PCG -- test infrastructure, never imported by the product path."""
