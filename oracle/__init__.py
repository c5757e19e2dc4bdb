"""Serial CPU oracle for TPC track-model encoding/decoding (test infrastructure only)."""
